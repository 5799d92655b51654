"""High-precision scalar expansions of the paper's schemes (test helper).

Each factorised scheme of Sec. 2.1 is a polynomial in A; here it is expanded
in mpmath from the coefficients printed in the paper (``golden/paper_tables.json``)
so that tests can (i) check those coefficients against the Taylor series of
cos and sin, (ii) recompute the admissible norms theta_2m of Tables 1-2 from
the error series of Sec. 3, and (iii) compare the oracle's polynomial, read off
a nilpotent shift matrix, coefficient by coefficient.
"""
from __future__ import annotations

import json
import os
from functools import lru_cache

import mpmath as mp

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
mp.mp.dps = 60


def tables():
    with open(os.path.join(GOLDEN, "paper_tables.json")) as f:
        return json.load(f)


def _add(*ps):
    n = max(len(p) for p in ps)
    r = [mp.mpf(0)] * n
    for p in ps:
        for i, c in enumerate(p):
            r[i] += c
    return r


def _mul(p, q):
    r = [mp.mpf(0)] * (len(p) + len(q) - 1)
    for i, a in enumerate(p):
        if a == 0:
            continue
        for j, b in enumerate(q):
            r[i + j] += a * b
    return r


def _sc(c, p):
    return [c * x for x in p]


def cos_taylor(k: int):
    return mp.mpf(-1) ** (k // 2) / mp.factorial(k) if k % 2 == 0 else mp.mpf(0)


def sin_taylor(k: int):
    return mp.mpf(-1) ** ((k - 1) // 2) / mp.factorial(k) if k % 2 == 1 else mp.mpf(0)


def _k7_parts(a):
    I, X = [mp.mpf(1)], [mp.mpf(0), mp.mpf(1)]
    A2 = _mul(X, X)
    A4 = _mul(A2, A2)
    A6 = _mul(A4, A2)
    Cj = {j: _add(_sc(a[(0, j)], I), _sc(a[(1, j)], A2), _sc(a[(2, j)], A4), _sc(a[(3, j)], A6))
          for j in (1, 2, 3, 4)}
    A12 = _add(Cj[3], _mul(Cj[4], Cj[4]))
    T24 = _add(Cj[1], _mul(_add(Cj[2], A12), A12))
    return A2, A4, A6, A12, T24


def _k7_sine(z, parts):
    I, X = [mp.mpf(1)], [mp.mpf(0), mp.mpf(1)]
    A2, A4, A6, A12, T24 = parts
    C48 = _mul(_add(_sc(z[6], I), _sc(z[7], A2), _sc(z[8], A4), _sc(z[9], A6),
                    _sc(z[10], A12), _sc(z[11], T24)), T24)
    return _mul(X, _add(_sc(z[0], I), _sc(z[1], A2), _sc(z[2], A4), _sc(z[3], A6),
                        _sc(z[4], A12), _sc(z[5], T24), C48))


_A_KEYS = [(2, 1), (3, 1), (0, 2), (1, 2), (2, 2), (3, 2), (0, 3), (1, 3), (2, 3), (3, 3),
           (1, 4), (2, 4), (3, 4)]
_Z_FREE = [0, 1, 2, 3, 4, 5, 7, 8, 9, 10, 11]


def _newton(fun, x, steps=5):
    """Newton's method with a forward-difference Jacobian (square systems)."""
    n = len(x)
    for _ in range(steps):
        f = fun(x)
        J = mp.matrix(n, n)
        h = mp.mpf(10) ** -35
        for j in range(n):
            x2 = list(x)
            x2[j] += h
            f2 = fun(x2)
            for i in range(n):
                J[i, j] = (f2[i] - f[i]) / h
        d = mp.lu_solve(J, mp.matrix(f))
        x = [x[i] - d[i] for i in range(n)]
    return x


@lru_cache(maxsize=None)
def schemes(refined: bool = False):
    """Coefficient lists (index = power of A) of every approximant.

    Keys: 'c4', 's5', 'c8', 's79', 's9', 'c16', 's17', 'c24', 's23'.
    With ``refined`` the k = 7 coefficients (printed to 20 digits) are
    polished by Newton's method on the equations they solve: the cosine
    matches cos through A^24 (13 equations, 13 unknowns) and the sine, with
    z6 = 1, matches sin through A^21 (11 equations, 11 unknowns).
    """
    T = tables()
    I, X = [mp.mpf(1)], [mp.mpf(0), mp.mpf(1)]
    A2 = _mul(X, X)
    A4 = _mul(A2, A2)
    f = mp.factorial
    out = {}
    # k = 3: eqs. Algorithm3cA, Algorithm3sA
    out["c4"] = _add(I, _sc(-1 / f(2), A2), _sc(1 / f(4), A4))
    out["s5"] = _mul(X, _add(I, _sc(-1 / f(3), A2), _sc(1 / f(5), A4)))
    # k = 4: eqs. Algorithm4cA, Algorithm4sA, Algorithm5sA
    A8 = _mul(A4, _add(_sc(-1 / f(6), A2), _sc(1 / f(8), A4)))
    out["c8"] = _add(I, _sc(-1 / f(2), A2), _sc(1 / f(4), A4), A8)
    out["s79"] = _mul(X, _add(I, _sc(-1 / f(3), A2), _sc(1 / f(5), A4), _sc(f(6) / f(7), A8)))
    A8b = _mul(A4, _add(_sc(-1 / f(7), A2), _sc(1 / f(9), A4)))
    out["s9"] = _mul(X, _add(I, _sc(-1 / f(3), A2), _sc(1 / f(5), A4), A8b))
    # k = 6: eqs. Algorithm6cA, cosm8, Algorithm6sA
    r = mp.sqrt(36681)
    x = {k: mp.mpf(eval(v, {"r": r, "__builtins__": {}}, {})) if "r" in v else mp.mpf(mp.fraction(*map(int, v.split("/"))))
         for k, v in T["k6_x"].items() if not k.startswith("_")}
    z6 = [mp.mpf(mp.fraction(*map(int, s.split("/")))) for s in T["k6_z"]["z"]]
    A8 = _mul(A4, _add(_sc(x["x1"], A2), _sc(x["x2"], A4)))
    A16 = _mul(_add(_sc(x["x3"], A4), A8),
               _add(_sc(x["x4"], I), _sc(x["x5"], A2), _sc(x["x6"], A4), _sc(x["x7"], A8)))
    T16 = _add(I, _sc(mp.mpf(-1) / 2, A2), _sc(x["x8"], A4), A16)
    out["c16"] = T16
    C24 = _mul(_add(_sc(z6[5], I), _sc(z6[5], A2), _sc(z6[6], A4), _sc(z6[7], A8), _sc(z6[8], T16)), A8)
    out["s17"] = _mul(X, _add(_sc(z6[0], I), _sc(z6[1], A2), _sc(z6[2], A4), _sc(z6[3], A8),
                              _sc(z6[4], T16), C24))
    # k = 7: eqs. Algorithm7cA + Coefs7cA, Algorithm7sA + Coefs7sA
    a = {tuple(int(t) for t in k.split(",")): mp.mpf(v) for k, v in T["k7_a"].items()
         if not k.startswith("_")}
    z7 = [mp.mpf(s) for s in T["k7_z"]["z"]]
    if refined:
        def fc(av):
            aa = dict(a)
            aa.update(zip(_A_KEYS, av))
            T24 = _k7_parts(aa)[4]
            return [T24[2 * i] - cos_taylor(2 * i) for i in range(13)]
        av = _newton(fc, [a[k] for k in _A_KEYS])
        a.update(zip(_A_KEYS, av))
        parts = _k7_parts(a)

        def fs(zv):
            zz = list(z7)
            for i, v in zip(_Z_FREE, zv):
                zz[i] = v
            S = _k7_sine(zz, parts)
            return [S[2 * i + 1] - sin_taylor(2 * i + 1) for i in range(11)]
        zv = _newton(fs, [z7[i] for i in _Z_FREE])
        for i, v in zip(_Z_FREE, zv):
            z7[i] = v
    parts = _k7_parts(a)
    out["c24"] = parts[4]
    out["s23"] = _k7_sine(z7, parts)
    return out


def theta(poly, sine: bool, u, nterms: int = 150):
    """Largest theta with sum_k |alpha_k| theta^k <= u, alpha_k = taylor_k - poly_k,
    the series truncated after ``nterms`` powers (Sec. 3, eqs. newtyerrsertay and
    newtyerrnorm)."""
    tay = sin_taylor if sine else cos_taylor
    coeff = []
    for k in range(nterms + 1):
        pk = poly[k] if k < len(poly) else mp.mpf(0)
        coeff.append(abs(tay(k) - pk))
    lo, hi = mp.mpf(0), mp.mpf(20)
    for _ in range(120):
        mid = (lo + hi) / 2
        if sum(c * mid ** k for k, c in enumerate(coeff)) > u:
            hi = mid
        else:
            lo = mid
    return lo


# ------------------------------------------------------------- Sec. 2.2 ---
# The c(t^2 A), s(t, A) schemes are the Sec. 2.1 polynomials with A_2 = A^2
# replaced by B = t^2 A and the leading factor A of the sine replaced by t:
# their coefficients in B are the even coefficients of the cosine polynomial
# and the odd coefficients of the sine polynomial of the Sec. 2.1 scheme.
CS_SCHEMES = {0: ("c8", "s79"), 1: ("c8", "s9"), 2: ("c16", "s17"), 3: ("c24", "s23")}


def cs_coefficients(family: int, refined: bool = False):
    polys = schemes(refined=refined)
    ck, sk = CS_SCHEMES[family]
    pc, ps = polys[ck], polys[sk]
    cos_b = [pc[2 * k] if 2 * k < len(pc) else mp.mpf(0) for k in range(len(pc) // 2 + 1)]
    sin_b = [ps[2 * k + 1] if 2 * k + 1 < len(ps) else mp.mpf(0) for k in range(len(ps) // 2 + 1)]
    return cos_b, sin_b


def cos_b_taylor(k: int):
    return mp.mpf(-1) ** k / mp.factorial(2 * k)


def sin_b_taylor(k: int):
    return mp.mpf(-1) ** k / mp.factorial(2 * k + 1)


def theta_b(coef, target, u, nterms: int = 150):
    """Largest ||B|| with sum_k |target_k - coef_k| ||B||^k <= u (150 terms)."""
    c = []
    for k in range(nterms + 1):
        ck = coef[k] if k < len(coef) else mp.mpf(0)
        a = abs(target(k) - ck)
        c.append(a if a > mp.mpf(10) ** -45 else mp.mpf(0))
    lo, hi = mp.mpf(0), mp.mpf(400)
    for _ in range(160):
        mid = (lo + hi) / 2
        if sum(ci * mid ** k for k, ci in enumerate(c)) > u:
            hi = mid
        else:
            lo = mid
    return lo
