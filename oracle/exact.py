"""Exact rational checks for tiny systems -- TEST INFRASTRUCTURE ONLY.

Pure Python with ``fractions.Fraction``; meant for n <= ~12.

* ``ge_solve``: dense Gaussian elimination with row pivoting in exact
  rationals (the plain definition x = A^{-1} f and det A).
* ``lu_solve``: the R1/R2 recurrences (LU without pivoting, Sec. 1 of
  Veneva & Ayriyan) in exact rationals.
* ``symbolic_solve``: the R3 rule of the symbolic methods SPDM/STDM (Sec. 1:
  a zero pivot is replaced by a symbol t and the solution is taken at the
  limit t -> 0; Sec. 3.2 Remark 1: the determinant in O(N)), carried out with
  exact rational functions of t, so no truncation is involved.
"""
from fractions import Fraction


# ---------------------------------------------------------------- polynomials
def _trim(p):
    p = list(p)
    while p and p[-1] == 0:
        p.pop()
    return p


def padd(p, q):
    n = max(len(p), len(q))
    return _trim([(p[i] if i < len(p) else 0) + (q[i] if i < len(q) else 0) for i in range(n)])


def pneg(p):
    return [-v for v in p]


def pmul(p, q):
    if not p or not q:
        return []
    r = [Fraction(0)] * (len(p) + len(q) - 1)
    for i, u in enumerate(p):
        for j, v in enumerate(q):
            r[i + j] += u * v
    return _trim(r)


def pdivmod(p, q):
    p = _trim(p)
    q = _trim(q)
    if not q:
        raise ZeroDivisionError("polynomial division by zero")
    quo = [Fraction(0)] * max(len(p) - len(q) + 1, 1)
    rem = list(p)
    while len(rem) >= len(q) and rem:
        shift = len(rem) - len(q)
        coef = rem[-1] / q[-1]
        quo[shift] = coef
        for i, v in enumerate(q):
            rem[i + shift] -= coef * v
        rem = _trim(rem)
    return _trim(quo), rem


def pgcd(p, q):
    p, q = _trim(p), _trim(q)
    while q:
        _, r = pdivmod(p, q)
        p, q = q, r
    if not p:
        return [Fraction(1)]
    lead = p[-1]
    return [v / lead for v in p]


def peval0(p):
    return p[0] if p else Fraction(0)


# --------------------------------------------------------- rational functions
class RF:
    """num(t) / den(t), reduced, den monic."""

    __slots__ = ("num", "den")

    def __init__(self, num, den=None):
        num = _trim([Fraction(v) for v in num])
        den = _trim([Fraction(v) for v in (den if den is not None else [1])])
        if not den:
            raise ZeroDivisionError("rational function with zero denominator")
        if not num:
            self.num, self.den = [], [Fraction(1)]
            return
        g = pgcd(num, den)
        if len(g) > 1:
            num, _ = pdivmod(num, g)
            den, _ = pdivmod(den, g)
        lead = den[-1]
        self.num = [v / lead for v in num]
        self.den = [v / lead for v in den]

    @staticmethod
    def const(v):
        return RF([Fraction(v)])

    @staticmethod
    def symbol():
        return RF([Fraction(0), Fraction(1)])

    def is_zero(self):
        return not self.num

    def __add__(self, o):
        return RF(padd(pmul(self.num, o.den), pmul(o.num, self.den)), pmul(self.den, o.den))

    def __sub__(self, o):
        return RF(padd(pmul(self.num, o.den), pneg(pmul(o.num, self.den))), pmul(self.den, o.den))

    def __mul__(self, o):
        return RF(pmul(self.num, o.num), pmul(self.den, o.den))

    def __truediv__(self, o):
        if o.is_zero():
            raise ZeroDivisionError("division by the zero function")
        return RF(pmul(self.num, o.den), pmul(self.den, o.num))

    def at0(self):
        """Value at t = 0, or None for a pole."""
        d0 = peval0(self.den)
        if d0 == 0:
            return None
        return peval0(self.num) / d0


# ------------------------------------------------------------------ matrices
def dense(k, a, b, c, d, e):
    n = len(c)
    A = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        A[i][i] = Fraction(c[i])
        if i >= 1:
            A[i][i - 1] = Fraction(b[i])
        if i + 1 < n:
            A[i][i + 1] = Fraction(d[i])
        if k == 2:
            if i >= 2:
                A[i][i - 2] = Fraction(a[i])
            if i + 2 < n:
                A[i][i + 2] = Fraction(e[i])
    return A


def ge_solve(A, f):
    """Exact Gaussian elimination with row pivoting.  Returns (x or None, det)."""
    n = len(A)
    M = [list(map(Fraction, row)) + [Fraction(f[i])] for i, row in enumerate(A)]
    det = Fraction(1)
    for j in range(n):
        p = next((i for i in range(j, n) if M[i][j] != 0), None)
        if p is None:
            return None, Fraction(0)
        if p != j:
            M[j], M[p] = M[p], M[j]
            det = -det
        det *= M[j][j]
        for i in range(j + 1, n):
            if M[i][j] != 0:
                l = M[i][j] / M[j][j]
                for cc in range(j, n + 1):
                    M[i][cc] -= l * M[j][cc]
    x = [Fraction(0)] * n
    for i in range(n - 1, -1, -1):
        s = M[i][n] - sum(M[i][cc] * x[cc] for cc in range(i + 1, n))
        x[i] = s / M[i][i]
    return x, det


def _recurrence(k, a, b, c, d, e, f, mk_const, on_zero_pivot):
    """The R1 (k=1) / R2 (k=2) recurrence over any field-like type.

    Returns (x, pivots).  ``on_zero_pivot(mu)`` decides what a zero pivot becomes.
    """
    n = len(c)
    zero = mk_const(0)
    alpha = [zero] * n
    beta = [zero] * n
    z = [zero] * n
    piv = []
    for i in range(n):
        ai = mk_const(a[i]) if (k == 2 and i >= 2) else zero
        g = mk_const(b[i]) if i >= 1 else zero
        if k == 2 and i >= 2:
            g = g - alpha[i - 2] * ai
        m = mk_const(c[i])
        if k == 2 and i >= 2:
            m = m - beta[i - 2] * ai
        if i >= 1:
            m = m - alpha[i - 1] * g
        m = on_zero_pivot(m)
        piv.append(m)
        if i <= n - 2:
            num = mk_const(d[i])
            if k == 2 and i >= 1:
                num = num - beta[i - 1] * g
            alpha[i] = num / m
        if k == 2 and i <= n - 3:
            beta[i] = mk_const(e[i]) / m
        zi = mk_const(f[i])
        if k == 2 and i >= 2:
            zi = zi - z[i - 2] * ai
        if i >= 1:
            zi = zi - z[i - 1] * g
        z[i] = zi / m
    x = [zero] * n
    for i in range(n - 1, -1, -1):
        xi = z[i]
        if i + 1 < n:
            xi = xi - alpha[i] * x[i + 1]
        if k == 2 and i + 2 < n:
            xi = xi - beta[i] * x[i + 2]
        x[i] = xi
    return x, piv


def lu_solve(k, a, b, c, d, e, f):
    """R1/R2 in exact rationals.  Raises ZeroDivisionError on a zero pivot."""

    def check(m):
        if m == 0:
            raise ZeroDivisionError("zero pivot")
        return m

    x, _ = _recurrence(k, a, b, c, d, e, f, Fraction, check)
    return x


def symbolic_solve(k, a, b, c, d, e, f):
    """R3 with exact rational functions of t.

    Returns dict(x=[Fraction or None], det=Fraction, nflag=int, status=str);
    status is "OK" or "SINGULAR".
    """
    flags = [0]

    def rule(m):
        if m.is_zero():
            flags[0] += 1
            return RF.symbol()
        return m

    x, piv = _recurrence(k, a, b, c, d, e, f, RF.const, rule)
    det = RF.const(1)
    for m in piv:
        det = det * m
    det0 = det.at0()
    xs = [v.at0() for v in x]
    status = "SINGULAR" if (det0 is None or det0 == 0) else "OK"
    return dict(x=xs, det=det0 if det0 is not None else Fraction(0), nflag=flags[0],
                status=status)
