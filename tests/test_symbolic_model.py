"""CPU checks of the model of the GPU symbolic fix-up's arithmetic (symbolic_model.py,
a lane-by-lane restatement of csrc/symbolic.cuh) against exact rational functions of t
(oracle.exact) on integer systems with crowded zero pivots: the same acceptance bar as
the GPU test -- the exact limit with status OK, SINGULAR for a singular matrix, and
SYMBOLIC_RANGE (the window or the precision ran out) on at most 1 % -- so that a change
of the kernel's series arithmetic can be checked here before it reaches a GPU."""
import numpy as np
import pytest

import symbolic_model as M
from oracle import exact

U = np.finfo(np.float64).eps / 2


@pytest.mark.parametrize("k", [1, 2])
def test_model_against_exact_crowded(k):
    rng = np.random.default_rng(700 + k)
    tally = dict(nonsingular=0, singular=0, range=0, singular_range=0)
    for _ in range(160):
        n = int(rng.integers(3, 13))
        pick = lambda vals: [int(v) for v in rng.choice(vals, n)]
        a, b, d, e, f = (pick([-2, -1, 0, 0, 1, 2]) for _ in range(5))
        c = pick([0, 0, 0, 1, -1])
        if k == 1:
            a, e = [0] * n, [0] * n
        sym = exact.symbolic_solve(k, a, b, c, d, e, f)
        if sym["nflag"] == 0:
            continue
        st, x, dm, dex = M.solve(k, a, b, c, d, e, f)
        if sym["status"] == "SINGULAR":
            tally["singular"] += 1
            assert st in (M.SINGULAR, M.RANGE), st
            tally["singular_range"] += st == M.RANGE
            continue
        tally["nonsingular"] += 1
        if st == M.RANGE:
            tally["range"] += 1
            continue
        assert st == M.OK
        xe = np.array([float(v) for v in sym["x"]])
        kappa = np.linalg.cond(np.array(exact.dense(k, a, b, c, d, e), dtype=float), np.inf)
        assert np.abs(np.array(x) - xe).max() <= 1e3 * kappa * U * max(1.0, np.abs(xe).max())
        assert abs(dm * 2.0 ** dex - float(sym["det"])) <= 1e-9 * abs(float(sym["det"]))
    assert tally["nonsingular"] >= 10 and tally["singular"] >= 10
    assert tally["range"] <= max(1, tally["nonsingular"] // 100), tally
    assert tally["singular_range"] <= max(1, tally["singular"] // 100), tally


def test_model_window_bookkeeping():
    """A single zero pivot (TD [[0, 1], [1, 0]] within a larger system) needs t^1 at most:
    the first pass settles it; the determinant is the exact one."""
    a = [0, 0, 0, 0]
    b = [0, 1, 1, 1]
    c = [0, 0, 2, 2]
    d = [1, 1, 1, 0]
    e = [0, 0, 0, 0]
    f = [1, 2, 3, 4]
    st, x, V, mant, ex = M.attempt(1, *[[float(v) for v in arr] for arr in (a, b, c, d, e, f)],
                                   M.FIRST_E)
    sym = exact.symbolic_solve(1, a, b, c, d, e, f)
    assert st == M.OK and V == 0
    assert np.allclose(x, [float(v) for v in sym["x"]], rtol=0, atol=1e-15)
    assert mant * 2.0 ** ex == float(sym["det"])


def test_model_first_pass_settles_one_pd_zero_pivot():
    """PD rows with one exact zero pivot (a = b = c = 0 on row 7 of integer rows): the
    pole rows' products cost the known range two orders, so t^3 is the least first pass
    that still knows x to t^0 (t^2 runs out of window); the result is the exact limit."""
    n, j = 16, 7
    a = [0, 0] + [1] * (n - 2)
    b = [0] + [-3] * (n - 1)
    c = [9] * n
    d = [-3] * (n - 1) + [0]
    e = [1] * (n - 2) + [0, 0]
    a[j] = b[j] = c[j] = 0
    f = [(3 * i) % 7 - 3 for i in range(n)]
    rows = [[float(v) for v in arr] for arr in (a, b, c, d, e, f)]
    assert M.FIRST_E == 3
    assert M.attempt(2, *rows, 2)[0] == M.RANGE
    st, x, V, mant, ex = M.attempt(2, *rows, M.FIRST_E)
    sym = exact.symbolic_solve(2, a, b, c, d, e, f)
    assert st == M.OK and V == 0 and sym["status"] == "OK"
    xs = np.array([float(v) for v in sym["x"]])
    assert np.abs(np.array(x) - xs).max() <= 1e-13 * np.abs(xs).max()
