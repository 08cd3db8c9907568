"""A CPU model of the GPU symbolic fix-up's arithmetic (csrc/symbolic.cuh), for tests.

It mirrors the kernel operation for operation: one series is a list of 32 lane values
(lane l holds the coefficient of t^(l - 15)) in double-double, with the kernel's
known-range bookkeeping (hi, v, top), residue flush, compensated sums of products,
long division by three numerators at once, the positive extents 3 then 16, and the
status rules.  Fused multiply-adds are evaluated exactly and rounded once (through
fractions), as the GPU's FMA does.  It is test infrastructure: it lets the series
pass be checked on the CPU against exact rational functions, and a disagreement
between it and the GPU points at the kernel's code rather than at its arithmetic.
It holds none of the oracle's code.
"""
import math
from fractions import Fraction

KZ = 15
KMAXE = 31 - KZ
FIRST_E = 3
NONE = 1 << 20
RESIDUE = 2.0 ** -80
OK, SINGULAR, NONFINITE, RANGE = 0, 4, 5, 7


def fma(a, b, c):
    if not (math.isfinite(a) and math.isfinite(b) and math.isfinite(c)):
        return a * b + c
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def two_sum(a, b):
    s = a + b
    bv = s - a
    av = s - bv
    return s, (a - av) + (b - bv)


def fast_two_sum(a, b):
    s = a + b
    return s, b - (s - a)


def dd_add(x, y):
    sh, sl = two_sum(x[0], y[0])
    th, tl = two_sum(x[1], y[1])
    sh, sl = fast_two_sum(sh, sl + th)
    return fast_two_sum(sh, sl + tl)


def dd_mul(x, y):
    p = x[0] * y[0]
    e = fma(x[0], y[0], -p)
    e = fma(x[0], y[1], e)
    e = fma(x[1], y[0], e)
    return fast_two_sum(p, e)


def dd_mul_d(x, s):
    p = x[0] * s
    e = fma(x[0], s, -p)
    e = fma(x[1], s, e)
    return fast_two_sum(p, e)


def dd_recip(y):
    r0 = 1.0 / y[0]
    res = dd_add((1.0, 0.0), tuple(-v for v in dd_mul_d(y, r0)))
    return fast_two_sum(r0, r0 * res[0])


class Acc:
    def __init__(self, x=(0.0, 0.0)):
        self.s, self.c, self.mag = x[0], x[1], abs(x[0])

    def fma(self, x, y, sign):
        p = x[0] * y[0]
        pe = fma(x[0], y[0], -p)
        pe = fma(x[0], y[1], pe)
        pe = fma(x[1], y[0], pe)
        th, tl = two_sum(self.s, sign * p)
        self.s = th
        self.c = self.c + fma(sign, pe, tl)
        self.mag = self.mag + abs(p)

    def value(self):
        v = two_sum(self.s, self.c)
        if abs(v[0]) <= RESIDUE * self.mag:
            return (0.0, 0.0)
        return v


class Ser:
    def __init__(self, q, hi, v=None, top=None):
        self.q = list(q)
        self.hi = hi
        if v is None:
            self.set_meta()
        else:
            self.v, self.top = v, top

    def set_meta(self):
        for lane in range(32):
            if lane - KZ >= self.hi:
                self.q[lane] = (0.0, 0.0)
        nz = [lane for lane in range(32) if self.q[lane][0] != 0.0]
        self.v = nz[0] - KZ if nz else NONE
        self.top = nz[-1] - KZ if nz else -NONE


ZERO = (0.0, 0.0)


def veff(s):
    return s.v if s.v != NONE else s.hi


def constant(x, E):
    q = [ZERO] * 32
    q[KZ] = (x, 0.0)
    nz = x != 0.0
    return Ser(q, E + 1, 0 if nz else NONE, 0 if nz else -NONE)


def symbol(E):
    q = [ZERO] * 32
    q[KZ + 1] = (1.0, 0.0)
    return Ser(q, E + 1, 1, 1)


def sub(x, y):
    q = []
    for lane in range(32):
        d = dd_add(x.q[lane], (-y.q[lane][0], -y.q[lane][1]))
        if abs(d[0]) <= RESIDUE * (abs(x.q[lane][0]) + abs(y.q[lane][0])):
            d = ZERO
        q.append(d)
    return Ser(q, min(x.hi, y.hi))


def sub_scaled(x, y, s, E):
    vs = 0 if s != 0.0 else E + 1
    p = Ser([dd_mul_d(y.q[lane], s) for lane in range(32)],
            min(E + 1, min(veff(y) + E + 1, vs + y.hi)))
    return sub(x, p)


def mul(x, y, E, err):
    hi = min(E + 1, min(veff(x) + y.hi, veff(y) + x.hi))
    if x.v == NONE or y.v == NONE:
        return Ser([ZERO] * 32, hi)
    if x.v + y.v < -KZ:
        err[0] = True
    u, w = (y, x) if (x.top - x.v) > (y.top - y.v) else (x, y)
    q = []
    for lane in range(32):
        e = lane - KZ
        a = Acc()
        live = e < hi
        for i in range(u.v, u.top + 1):
            j = e - i
            if live and w.v <= j <= w.top:
                a.fma(u.q[i + KZ], w.q[j + KZ], 1.0)
        q.append(a.value() if live else ZERO)
    return Ser(q, hi)


def div3(num, use, m, E, err):
    out = [None, None, None]
    if m.v == NONE:
        err[0] = True
        return [Ser([ZERO] * 32, -KZ) for _ in range(3)]
    vm = m.v
    inv = dd_recip(m.q[vm + KZ])
    v, hi, act, lim = [0] * 3, [E + 1] * 3, [False] * 3, [0] * 3
    acc = [[Acc() for _ in range(32)] for _ in range(3)]
    res = [[ZERO] * 32 for _ in range(3)]
    steps = 0
    for k in range(3):
        if not use[k]:
            continue
        if num[k].v == NONE:
            hi[k] = min(E + 1, num[k].hi - vm)
            continue
        v[k] = num[k].v - vm
        hi[k] = min(E + 1, v[k] + min(num[k].hi - num[k].v, m.hi - vm))
        if v[k] < -KZ:
            err[0] = True
            continue
        act[k] = True
        for lane in range(32):
            e = lane - KZ
            if v[k] <= e < hi[k]:
                acc[k][lane] = Acc(num[k].q[e + vm + KZ])
        lim[k] = hi[k] - v[k]
        if m.top == vm:          # a monomial divisor: the quotient ends at n's top
            lim[k] = min(lim[k], num[k].top - num[k].v + 1)
        steps = max(steps, lim[k])
    for st in range(steps):
        for k in range(3):
            if not act[k] or st >= lim[k]:
                continue
            ek = v[k] + st
            c = dd_mul(acc[k][ek + KZ].value(), inv)
            res[k][ek + KZ] = c
            for lane in range(32):
                e = lane - KZ
                j = e - ek
                if j >= 1 and e < hi[k] and vm + j <= m.top:
                    acc[k][lane].fma(m.q[vm + j + KZ], c, -1.0)
    for k in range(3):
        out[k] = Ser(res[k], hi[k])
    return out


def frexp_mul(mant, ex, lead):
    m, e2 = math.frexp(lead)
    mant *= m
    ex += e2
    mant, e3 = math.frexp(mant)
    return mant, ex + e3


def attempt(k, a, b, c, d, e, f, E, want_x=True):
    """One pass with positive extent E.  Returns (status, x, V, mant, ex)."""
    n = len(c)
    err = [False]
    V, mant, ex = 0, 1.0, 0
    AL, BE, Z = [None] * n, [None] * n, [None] * n
    zero = constant(0.0, E)
    al1 = al2 = be1 = be2 = z1 = z2 = zero
    for i in range(n):
        if err[0]:
            break
        ai = a[i] if (k == 2 and i >= 2) else 0.0
        g = constant(b[i] if i >= 1 else 0.0, E)
        if k == 2 and i >= 2:
            g = sub_scaled(g, al2, ai, E)
        m = constant(c[i], E)
        if k == 2 and i >= 2:
            m = sub_scaled(m, be2, ai, E)
        if i >= 1:
            m = sub(m, mul(al1, g, E, err))
        if m.v == NONE:
            if m.hi < 1:
                err[0] = True
            m = symbol(E)
        V += m.v
        mant, ex = frexp_mul(mant, ex, m.q[(m.v + KZ) & 31][0])
        num = [constant(0.0, E), None, constant(0.0, E)]
        use = [i + 1 < n, k == 2 and i + 2 < n, want_x]
        if use[0]:
            num[0] = constant(d[i], E)
            if k == 2 and i >= 1:
                num[0] = sub(num[0], mul(be1, g, E, err))
        num[1] = constant(e[i] if use[1] else 0.0, E)
        if want_x:
            num[2] = constant(f[i], E)
            if k == 2 and i >= 2:
                num[2] = sub_scaled(num[2], z2, ai, E)
            if i >= 1:
                num[2] = sub(num[2], mul(z1, g, E, err))
        r = div3(num, use, m, E, err)
        if not use[0]:
            r[0] = constant(0.0, E)
        if not use[1]:
            r[1] = constant(0.0, E)
        AL[i], BE[i], Z[i] = r
        al2, al1 = al1, r[0]
        be2, be1 = be1, r[1]
        z2, z1 = z1, r[2]
    x = [float("nan")] * n
    status = OK
    if not err[0] and want_x:
        x1 = x2 = constant(0.0, E)
        bad = False
        for i in range(n - 1, -1, -1):
            if err[0]:
                break
            xi = Z[i]
            if i + 1 < n:
                xi = sub(xi, mul(AL[i], x1, E, err))
            if k == 2 and i + 2 < n:
                xi = sub(xi, mul(BE[i], x2, E, err))
            q = [ZERO if lane < KZ else xi.q[lane] for lane in range(32)]
            xi = Ser(q, xi.hi)
            if xi.hi <= 0:
                err[0] = True
            x[i] = xi.q[KZ][0]
            bad |= not math.isfinite(x[i])
            x2, x1 = x1, xi
        if bad:
            status = NONFINITE
    if err[0] or V < 0:
        status = RANGE
    elif V > 0:
        status = SINGULAR
    return status, x, V, mant, ex


def solve(k, a, b, c, d, e, f, want_x=True):
    """The fix-up of one system: extent 3, then 16 if that ran out of window.
    Returns (status, x, det_mant, det_exp)."""
    a, b, c, d, e, f = ([float(v) for v in arr] for arr in (a, b, c, d, e, f))
    st, x, V, mant, ex = attempt(k, a, b, c, d, e, f, FIRST_E, want_x)
    if st == RANGE:
        st, x, V, mant, ex = attempt(k, a, b, c, d, e, f, KMAXE, want_x)
    ok = st in (OK, NONFINITE) and V == 0
    return st, x, (mant if ok else 0.0), (ex if ok else 0)
