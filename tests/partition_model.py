"""A numpy model of the partitioned schedule's arithmetic (test infrastructure only).

It restates, for checking on the CPU, what the partitioned kernels compute: chunk k of
P restarts NPDM's recurrence at its first row and carries f and the coupling columns
B_k (through the forward sweep) and C_k (formed at the end); a first backward sweep
keeps the top and bottom K rows of g = A_k^-1 f_k, V = A_k^-1 B_k, W = A_k^-1 C_k in
the exchange slots (g, V1, W1, V2, W2 at 0, 2K, 4K, 6K, 8K); the block-tridiagonal
interface y_k + L_k y_{k-1} + U_k y_{k+1} = g_k is eliminated top-down over chunks
0 .. P/2-1 and bottom-up over P-1 .. P/2 on the mirrored system (slot of row r:
(r + K) mod 2K), the two halves meet in a 2K x 2K system, each half is
back-substituted, and each chunk is swept back once more with z - z_V u - z_W v.
The pivot guard treats a chunk pivot whose binary exponent lies 17 or more below that
of its row's largest entry, or an interface K x K block (or the meeting's Schur
complement) as close to singular, like a zero pivot.  Vectorised over systems; the
small solves use numpy's partially pivoted LU instead of the kernels' own, so results
agree with the kernels to rounding, not bit for bit.  Shares nothing with the CUDA
sources and is not the oracle: the oracle defines what a solve must return, this
model only reproduces how the partitioned schedule gets there.
"""
import numpy as np

TINY = 17


def _bexp(v):
    """IEEE binary64 biased exponent of |v| (0 for zero)."""
    _, e = np.frexp(np.abs(v))
    return np.where(v == 0, 0, e + 1022)


def _near_singular(A):
    """A: (..., K, K).  |det A| 17 binary orders per row below max(1, max|A_ij|)^K."""
    K = A.shape[-1]
    one = _bexp(np.float64(1.0))
    s = np.maximum(one, _bexp(A).reshape(A.shape[:-2] + (-1,)).max(-1))
    det = A[..., 0, 0] if K == 1 else A[..., 0, 0] * A[..., 1, 1] - A[..., 0, 1] * A[..., 1, 0]
    return (det == 0) | ((_bexp(det) - one) + K * TINY <= K * (s - one))


def solve(A, K, P, guard=True):
    """A: dict of (n, nsys) arrays a, b, c, d, e, f (a, e ignored for K = 1).
    Returns (x (n, nsys), failed (nsys,) bool): the systems the kernels would redo
    (their x is NaN here)."""
    n, ns = A["c"].shape
    NB, PW = 2 * K, 2 * K + 4 * K * K
    L0, rem = divmod(n, P)
    ks = np.arange(P)
    Ls = L0 + (ks < rem)
    s0 = ks * L0 + np.minimum(ks, rem)
    Lmax = int(Ls.max())
    z = lambda: np.zeros((P, ns))
    get = lambda q, i, mask: np.where(mask[:, None], A[q][np.clip(i, 0, n - 1)], 0.0)
    al, be, zf, zv1, zv2 = (np.zeros((Lmax, P, ns)) for _ in range(5))
    al1, al2, be1, be2, zf1, zf2, v11, v12, v21, v22 = (z() for _ in range(10))
    rc_last, rc_last2, g_last, d_last, e_last, e_last2 = (z() for _ in range(6))
    fail = np.zeros(ns, bool)
    with np.errstate(all="ignore"):
        for j in range(Lmax):
            live = (j < Ls)[:, None]
            i = s0 + j
            ag = get("a", i, (i >= 2) & (K == 2))
            bg = get("b", i, i >= 1)
            dg = get("d", i, i + 1 < n)
            eg = get("e", i, (i + 2 < n) & (K == 2))
            cc = A["c"][np.clip(i, 0, n - 1)]
            ff = A["f"][np.clip(i, 0, n - 1)]
            aa = ag if j >= 2 else 0 * ag
            bb = bg if j >= 1 else 0 * bg
            dd = np.where((j + 1 < Ls)[:, None], dg, 0.0)
            ee = np.where((j + 2 < Ls)[:, None], eg, 0.0)
            if K == 2:
                rv1 = ag if j == 0 else 0 * ag
                rv2 = bg if j == 0 else (ag if j == 1 else 0 * ag)
                g = bb - al2 * aa
                m = cc - be2 * aa - al1 * g
            else:
                rv1, rv2 = (bg if j == 0 else 0 * bg), 0 * bg
                g = bb
                m = cc - al1 * g
            ex = np.maximum.reduce([_bexp(v) for v in (cc, bg, dg, ag, eg)])
            trip = (m == 0) | (guard & (_bexp(m) + TINY <= ex)) if guard else (m == 0)
            fail |= (live & trip).any(0)
            rc = 1.0 / m
            alv = ((dd - be1 * g) if K == 2 else dd) * rc
            bev = ee * rc
            zfv = (ff - zf2 * aa - zf1 * g) * rc
            z1 = (rv1 - v12 * aa - v11 * g) * rc
            z2 = (rv2 - v22 * aa - v21 * g) * rc
            upd = lambda old, new: np.where(live, new, old)
            al[j], be[j], zf[j], zv1[j], zv2[j] = alv, bev, zfv, z1, z2
            al2, al1 = upd(al2, al1), upd(al1, alv)
            be2, be1 = upd(be2, be1), upd(be1, bev)
            zf2, zf1 = upd(zf2, zf1), upd(zf1, zfv)
            v12, v11 = upd(v12, v11), upd(v11, z1)
            v22, v21 = upd(v22, v21), upd(v21, z2)
            rc_last2, e_last2 = upd(rc_last2, rc_last), upd(e_last2, e_last)
            rc_last, g_last, d_last, e_last = upd(rc_last, rc), upd(g_last, g), upd(d_last, dg), upd(e_last, eg)
        # forward values of C's columns in the last K rows
        if K == 2:
            w12 = e_last2 * rc_last2
            w11 = (d_last - w12 * g_last) * rc_last
            w21 = e_last * rc_last
        else:
            w12, w11, w21 = 0 * rc_last, d_last * rc_last, 0 * rc_last
        zw1, zw2 = np.zeros((Lmax, P, ns)), np.zeros((Lmax, P, ns))
        for k in range(P):
            L = Ls[k]
            zw1[L - 1, k], zw2[L - 1, k] = w11[k], w21[k]
            if K == 2:
                zw1[L - 2, k] = w12[k]

        def back(zcol):
            """U^-1 zcol per chunk: (Lmax, P, ns)."""
            x = np.zeros_like(zcol)
            x1, x2 = z(), z()
            for j in range(Lmax - 1, -1, -1):
                live = (j < Ls)[:, None]
                v = zcol[j] - al[j] * x1 - (be[j] * x2 if K == 2 else 0)
                x[j] = np.where(live, v, 0.0)
                x2, x1 = np.where(live, x1, x2), np.where(live, v, x1)
            return x

        cols = [back(zf), back(zv1), back(zw1)] + ([back(zv2), back(zw2)] if K == 2 else [])
        xch = np.zeros((P, PW, ns))
        for k in range(P):
            rows = list(range(K)) + list(range(Ls[k] - K, Ls[k]))
            for ci, col in enumerate(cols):
                xch[k, ci * NB:(ci + 1) * NB] = col[rows, k]

        def eliminate(up):
            bad = np.zeros(ns, bool)
            rot = K if up else 0
            offP, offN = (2 * NB, NB) if up else (NB, 2 * NB)
            row = [(r + rot) % NB for r in range(NB)]
            for q in range(P // 2):
                kk = P - 1 - q if up else q
                e_ = xch[kk]
                R = np.zeros((ns, NB, K + 1))
                X = np.zeros((ns, NB, K))
                for r in range(NB):
                    R[:, r, K] = e_[row[r]]
                    R[:, r, 0] = e_[offN + row[r]]
                    if K == 2:
                        R[:, r, 1] = e_[offN + 2 * NB + row[r]]
                if q > 0:
                    ep = xch[kk + 1] if up else xch[kk - 1]
                    for r in range(NB):
                        vr = [e_[offP + row[r]]] + ([e_[offP + 2 * NB + row[r]]] if K == 2 else [])
                        for m_ in range(K):
                            for c_ in range(K):
                                X[:, r, c_] += vr[m_] * ep[NB * (1 + c_) + row[K + m_]]
                            R[:, r, K] -= vr[m_] * ep[row[K + m_]]
                Ab = np.eye(K)[None] - X[:, :K, :]
                bad |= _near_singular(Ab) if guard else np.zeros(ns, bool)
                Ab = np.where(bad[:, None, None], np.eye(K)[None], Ab)
                Rt = np.linalg.solve(Ab, R[:, :K, :])
                R[:, K:, :] += X[:, K:, :] @ Rt
                R[:, :K, :] = Rt
                for r in range(NB):
                    e_[row[r]] = R[:, r, K]
                    for c_ in range(K):
                        e_[NB * (1 + c_) + row[r]] = R[:, r, c_]
            return bad

        fail |= eliminate(False) | eliminate(True)
        mid = P // 2
        a_, b_ = xch[mid - 1], xch[mid]
        M = np.zeros((ns, NB, NB))
        rhs = np.zeros((ns, NB))
        for r in range(K):
            for c_ in range(K):
                M[:, r, c_] = float(r == c_)
                M[:, r, K + c_] = a_[NB * (1 + c_) + K + r]
                M[:, K + r, c_] = b_[NB * (1 + c_) + r]
                M[:, K + r, K + c_] = float(r == c_)
            rhs[:, r], rhs[:, K + r] = a_[K + r], b_[r]
        S = np.eye(K)[None] - M[:, K:, :K] @ M[:, :K, K:]
        if guard:
            fail |= _near_singular(S)
        M = np.where(fail[:, None, None], np.eye(NB)[None], M)
        uv = np.linalg.solve(M, rhs[..., None])[..., 0]
        u, v = uv[:, :K].T, uv[:, K:].T
        ya, yb = a_[:NB].copy(), b_[:NB].copy()
        for r in range(NB):
            for c_ in range(K):
                ya[r] -= a_[NB * (1 + c_) + r] * v[c_]
                yb[r] -= b_[NB * (1 + c_) + r] * u[c_]
        a_[:NB], b_[:NB] = ya, yb
        for up in (False, True):
            rot = K if up else 0
            for q in range(P // 2 - 2, -1, -1):
                kk = P - 1 - q if up else q
                e_, en = xch[kk], (xch[kk - 1] if up else xch[kk + 1])
                for r in range(NB):
                    sr = (r + rot) % NB
                    val = e_[sr].copy()
                    for c_ in range(K):
                        val -= e_[NB * (1 + c_) + sr] * en[(c_ + rot) % NB]
                    e_[sr] = val
        x = np.zeros((n, ns))
        for k in range(P):
            uk = xch[k - 1, K:NB] if k > 0 else np.zeros((K, ns))
            vk = xch[k + 1, :K] if k + 1 < P else np.zeros((K, ns))
            L = Ls[k]
            zz = zf[:L, k] - zv1[:L, k] * uk[0] - zw1[:L, k] * vk[0]
            if K == 2:
                zz = zz - zv2[:L, k] * uk[1] - zw2[:L, k] * vk[1]
            x1, x2 = np.zeros(ns), np.zeros(ns)
            for j in range(L - 1, -1, -1):
                xi = zz[j] - al[j, k] * x1 - (be[j, k] * x2 if K == 2 else 0)
                x[s0[k] + j] = xi
                x2, x1 = x1, xi
    x[:, fail] = np.nan
    return x, fail
