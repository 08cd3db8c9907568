"""Write zero_pivot_cases.json: hand-made systems with exact zero pivots.

Calls only the oracle (exact rational arithmetic, ``oracle.exact``).  Each case is
built so that LU without pivoting meets a pivot that is exactly 0 both in rational
and in IEEE arithmetic (all pivots before it are powers of two, so every earlier
quotient is exact), while A itself stays nonsingular -- the situation the symbolic
methods SPDM/STDM exist for (Veneva & Ayriyan, Sec. 1: the symbolic algorithms only
require nonsingularity).  Singular cases check the O(N) determinant (Sec. 3.2,
Remark 1).  The expected solution and determinant come from exact Gaussian
elimination with pivoting.

Run:  python tests/golden/make_zero_pivot_cases.py
"""
import json
import os
import random
import sys
from fractions import Fraction

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import exact  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "zero_pivot_cases.json")


def construct(k, n, flags, rng, consecutive=False):
    """Diagonals with exact zero pivots at the rows in `flags` (ints in [-2, 2])."""
    F = Fraction
    a = [F(rng.randint(-2, 2)) if (k == 2 and i >= 2) else F(0) for i in range(n)]
    b = [F(rng.randint(-2, 2)) if i >= 1 else F(0) for i in range(n)]
    d = [F(rng.randint(-2, 2)) if i <= n - 2 else F(0) for i in range(n)]
    e = [F(rng.randint(-2, 2)) if (k == 2 and i <= n - 3) else F(0) for i in range(n)]
    f = [F(rng.randint(-3, 3)) for i in range(n)]
    c = [F(0)] * n
    alpha = [F(0)] * n
    beta = [F(0)] * n
    first = min(flags)
    for i in range(n):
        if i > first:
            if consecutive and i == first + 1:
                # make gamma_{i} = 0 and mu_{i} = 0 as functions of t
                if k == 2:
                    a[i] = F(1)
                    b[i] = alpha[i - 2] * a[i]
                    c[i] = beta[i - 2] * a[i]
                else:
                    b[i] = F(0)
                    c[i] = F(0)
            else:
                c[i] = F(rng.choice([-3, -2, 2, 3, 5]))
            continue
        g = b[i] if i >= 1 else F(0)
        if k == 2 and i >= 2:
            g = g - alpha[i - 2] * a[i]
        s = F(0)
        if k == 2 and i >= 2:
            s += beta[i - 2] * a[i]
        if i >= 1:
            s += alpha[i - 1] * g
        if i in flags:
            c[i] = s
            continue
        p = F(rng.choice([1, -1, 2, -2]))
        c[i] = s + p
        num = d[i] - (beta[i - 1] * g if (k == 2 and i >= 1) else 0)
        alpha[i] = num / p if i <= n - 2 else F(0)
        beta[i] = e[i] / p if (k == 2 and i <= n - 3) else F(0)
    return a, b, c, d, e, f


def case_dict(name, k, diags, note):
    a, b, c, d, e, f = diags
    A = exact.dense(k, a, b, c, d, e)
    x, det = exact.ge_solve(A, f)
    sym = exact.symbolic_solve(k, a, b, c, d, e, f)
    s = lambda v: str(Fraction(v))
    return dict(name=name, k=k, n=len(c), note=note,
                a=[s(v) for v in a], b=[s(v) for v in b], c=[s(v) for v in c],
                d=[s(v) for v in d], e=[s(v) for v in e], f=[s(v) for v in f],
                x=None if x is None else [s(v) for v in x], det=s(det),
                nflag=sym["nflag"], status="OK" if det != 0 else "SINGULAR")


def main():
    cases = []
    # TD [[0, 1], [1, 0]]: the solution is f swapped
    cases.append(case_dict("td_swap", 1, ([0, 0], [0, 1], [0, 0], [1, 0], [0, 0], [3, 5]),
                           "c_0 = 0: the first pivot is zero; x = (f_1, f_0)"))
    specs = [("td_mid", 1, 7, [3], False), ("pd_mid", 2, 8, [4], False),
             ("pd_first", 2, 6, [0], False), ("pd_two_apart", 2, 10, [2, 6], False),
             ("pd_consecutive", 2, 9, [3], True), ("pd_near_end", 2, 7, [5], False),
             # two consecutive vanishing leading minors of a tridiagonal matrix force every
             # later minor to vanish (three-term recurrence), so this one must be SINGULAR
             ("td_consecutive_singular", 1, 8, [2], True)]
    for name, k, n, flags, consec in specs:
        want_singular = name.endswith("_singular")
        for seed in range(1, 500):
            rng = random.Random(1000 * seed + n)
            diags = construct(k, n, set(flags), rng, consecutive=consec)
            A = exact.dense(k, *diags[:5])
            x, det = exact.ge_solve(A, diags[5])
            if (det == 0) != want_singular:
                continue
            sym = exact.symbolic_solve(k, *diags)
            want = len(flags) + (1 if consec else 0)
            if sym["nflag"] < want:
                continue
            cases.append(case_dict(name, k, diags, "zero pivot(s) at rows %s%s" % (
                flags, " and the next row" if consec else "")))
            break
        else:
            raise RuntimeError("no case found for " + name)
    # exactly singular systems
    cases.append(case_dict("td_singular", 1, ([0, 0], [0, 1], [1, 1], [1, 0], [0, 0], [1, 2]),
                           "[[1, 1], [1, 1]]: det = 0"))
    cases.append(case_dict("pd_singular", 2,
                           ([0, 0, 1, 1], [0, 1, 2, 1], [1, 2, 3, 1], [1, 1, 1, 0], [1, 1, 0, 0],
                            [1, 2, 3, 4]),
                           "rows built so that det = 0"))
    with open(OUT, "w") as fh:
        json.dump(dict(citation="Veneva & Ayriyan, arXiv:1804.09666, Sec. 1 (symbolic methods "
                                "need only nonsingularity) and Sec. 3.2 Remark 1 (O(N) determinant); "
                                "values from exact rational Gaussian elimination",
                       generator="tests/golden/make_zero_pivot_cases.py", cases=cases), fh, indent=1)
    print("wrote", OUT, len(cases), "cases")


if __name__ == "__main__":
    main()
