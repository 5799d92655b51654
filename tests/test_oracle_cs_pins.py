"""Pins of the oracle's c(t^2 A), s(t, A) schemes (Sec. 2.2).

c(t^2 A) = cos(sqrt(t^2 A)) and s(t, A) = A^(-1/2) sin(sqrt(t^2 A)) are
pinned by: their coefficients in B = t^2 A read off a nilpotent shift matrix
against the Taylor series and the expanded printed coefficients; the
admissible norms recomputed from the Sec. 3 error series; the exponential
e^{tM}, M = [[0, I], [-A, 0]], whose blocks they are (Sec. 1, eq. symplectic);
eigendecompositions; double-angle identities; brute-force series.
"""
import math

import mpmath as mp
import numpy as np
import pytest

import oracle
import paper_poly as pp
from paper_2010_00465_gb300 import inputs

# family -> (cosine order in B, sine order in B) matched by the scheme
ORDERS = {0: (4, 3), 1: (4, 4), 2: (8, 8), 3: (12, 10)}
PRODUCTS = {0: 2, 1: 3, 2: 4, 3: 5}


def relfro(X, Y):
    return float(np.linalg.norm(X - Y) / max(np.linalg.norm(Y), 1e-300))


@pytest.mark.parametrize("family", [0, 1, 2, 3])
def test_coefficients_on_nilpotent_shift(family):
    cos_b, sin_b = pp.cs_coefficients(family)
    d = max(len(cos_b), len(sin_b)) + 1
    N = np.diag(np.ones(d - 1), 1)
    t = 0.75
    C, S, info = oracle.cs(N / t ** 2, t, family=family, sigma=0)   # B = N
    assert info["products"] == PRODUCTS[family]
    oc, os_ = ORDERS[family]
    for k in range(d):
        rc = float(cos_b[k]) if k < len(cos_b) else 0.0
        rs = float(sin_b[k]) if k < len(sin_b) else 0.0
        assert C[0, k] == pytest.approx(rc, rel=1e-13, abs=1e-300), ("cos", k)
        assert S[0, k] / t == pytest.approx(rs, rel=1e-13, abs=1e-300), ("sin", k)
    for k in range(oc + 1):
        assert C[0, k] == pytest.approx(float(pp.cos_b_taylor(k)), rel=1e-14, abs=0)
    for k in range(os_ + 1):
        assert S[0, k] / t == pytest.approx(float(pp.sin_b_taylor(k)), rel=1e-14, abs=0)


def test_printed_sign_of_p34_is_wrong():
    """Reading of eq. Algorithm83eA: with the printed '- (6!/7!) B_4' the B^3
    coefficient of P_{3,4}^s would be +1/7!; the series needs -1/7!."""
    b4_b3 = -1 / mp.factorial(6)            # B_4 = -B^3/6! + ...
    printed = -(mp.factorial(6) / mp.factorial(7)) * b4_b3
    corrected = +(mp.factorial(6) / mp.factorial(7)) * b4_b3
    assert printed == -pp.sin_b_taylor(3) and corrected == pp.sin_b_taylor(3)


@pytest.mark.slow
def test_theta_recomputed():
    for prec, u in (("double", mp.mpf(2) ** -53), ("single", mp.mpf(2) ** -24)):
        for f in range(4):
            cos_b, sin_b = pp.cs_coefficients(f, refined=True)
            th = min(pp.theta_b(cos_b, pp.cos_b_taylor, u), pp.theta_b(sin_b, pp.sin_b_taylor, u))
            got = oracle.cs_theta(prec, f)
            assert abs(float(th) - got) <= 6e-6 * got, (prec, f, float(th), got)


def test_cosine_theta_is_square_of_table():
    """The cosine parts are the Sec. 2.1 cosines in B = A^2, so their
    admissible ||B|| is theta_2m^2 of Tables 1-2 (recomputed)."""
    polys_cos = {0: 8, 1: 8, 2: 16, 3: 24}
    for f in range(4):
        cos_b, _ = pp.cs_coefficients(f, refined=True)
        th = float(pp.theta_b(cos_b, pp.cos_b_taylor, mp.mpf(2) ** -53))
        assert th == pytest.approx(oracle.theta("double", polys_cos[f], False) ** 2, rel=2e-4)


def test_selection():
    for prec in ("double", "single"):
        th = [oracle.cs_theta(prec, f) for f in range(4)]
        for nrm in np.geomspace(1e-8, 1e8, 201):
            f, sg = oracle.cs_select(nrm, prec)
            assert nrm / 4.0 ** sg <= th[f]
            assert sg == 0 or nrm / 4.0 ** (sg - 1) > th[f]
            for f2 in range(4):
                s2 = 0
                while nrm / 4.0 ** s2 > th[f2]:
                    s2 += 1
                assert PRODUCTS[f] + 2 * sg <= PRODUCTS[f2] + 2 * s2
    with pytest.raises(oracle.OracleError):
        oracle.cs_select(float("nan"))


def _eig_cs(A, t):
    w, V = np.linalg.eigh(A)
    r = np.sqrt(w.astype(complex))
    c = np.cos(t * r)
    s = np.where(np.abs(r) > 0, np.sin(t * r) / np.where(np.abs(r) > 0, r, 1), t)
    return ((V * c) @ V.T).real, ((V * s) @ V.T).real


@pytest.mark.parametrize("t", [0.1, 1.0, 3.0, 10.0])
@pytest.mark.parametrize("kind", ["psd", "indefinite"])
def test_symmetric_eigendecomposition(t, kind):
    X = inputs.matrix(16, "symmetric", 1.0, index=130)
    A = X @ X if kind == "psd" else X
    A = A * (4.0 / np.abs(A).sum(axis=0).max())
    C, S, info = oracle.cs(A, t)
    Cr, Sr = _eig_cs(A, t)
    tol = 1e-14 * (1 + 4.0 ** info["s"]) * max(1.0, np.abs(Cr).max())
    assert np.abs(C - Cr).max() <= tol
    assert np.abs(S - Sr).max() <= tol * max(1.0, t)


@pytest.mark.parametrize("family_name", ["normal", "triangular", "uniform01"])
@pytest.mark.parametrize("t", [0.3, 1.5, 6.0])
def test_exponential_blocks(family_name, t):
    """e^{tM}, M = [[0, I], [-A, 0]], has blocks [[c, s], [-A s, c]] (Sec. 1)."""
    sl = pytest.importorskip("scipy.linalg")
    n = 12
    A = inputs.matrix(n, family_name, 3.0, index=131)
    M = np.block([[np.zeros((n, n)), np.eye(n)], [-A, np.zeros((n, n))]])
    E = sl.expm(t * M)
    C, S, _ = oracle.cs(A, t)
    scale = max(1.0, np.abs(E).max())
    assert np.abs(C - E[:n, :n]).max() <= 1e-12 * scale
    assert np.abs(S - E[:n, n:]).max() <= 1e-12 * scale
    assert np.abs(-A @ S - E[n:, :n]).max() <= 1e-12 * scale
    assert np.abs(C - E[n:, n:]).max() <= 1e-12 * scale


def test_relation_to_cos_sin():
    """For A = X^2: c(t^2 A) = cos(tX) and s(t, A) X = sin(tX)."""
    X = inputs.matrix(10, "normal", 1.2, index=132)
    t = 1.7
    C, S, _ = oracle.cs(X @ X, t)
    Co, So, _ = oracle.cossin(t * X)
    assert relfro(C, Co) < 1e-13
    assert relfro(S @ X, So) < 1e-13


def test_double_angle_identities():
    A = inputs.matrix(14, "normal", 2.0, index=133)
    t = 1.1
    C, S, _ = oracle.cs(A, t)
    C2, S2, _ = oracle.cs(A, 2 * t)
    assert relfro(C2, 2 * C @ C - np.eye(14)) < 1e-12
    assert relfro(S2, 2 * S @ C) < 1e-12


def test_degenerate_cases():
    A = inputs.matrix(7, "normal", 5.0, index=134)
    C, S, _ = oracle.cs(A, 0.0)
    assert np.array_equal(C, np.eye(7)) and np.array_equal(S, np.zeros((7, 7)))
    C, S, _ = oracle.cs(np.zeros((7, 7)), 2.5)
    assert np.array_equal(C, np.eye(7)) and np.allclose(S, 2.5 * np.eye(7), rtol=0, atol=0)


@pytest.mark.parametrize("nrm", [0.01, 1.0, 10.0, 40.0])
def test_brute_force_series(nrm):
    mp.mp.dps = 60
    n = 5
    A = inputs.matrix(n, "normal", nrm, index=135)
    t = 0.9
    B = mp.matrix((t * t * A).tolist())
    P = mp.eye(n)
    Cs = mp.zeros(n, n)
    Ss = mp.zeros(n, n)
    for k in range(120):
        Cs += P * pp.cos_b_taylor(k)
        Ss += P * (t * pp.sin_b_taylor(k))
        P = P * B
    f = lambda X: np.array([[float(X[i, j]) for j in range(n)] for i in range(n)])
    C, S, _ = oracle.cs(A, t)
    assert relfro(C, f(Cs)) < 1e-13 and relfro(S, f(Ss)) < 1e-13


def _horner(coef, B):
    n = B.shape[0]
    P = float(coef[-1]) * np.eye(n)
    for c in reversed(coef[:-1]):
        P = P @ B + float(c) * np.eye(n)
    return P


@pytest.mark.parametrize("family", [0, 1, 2, 3])
def test_schemes_equal_expanded_polynomials(family):
    """c and s of each family equal their expanded polynomials in B = t^2 A
    (s times t) evaluated by Horner's rule, at sigma = 0 with ||B||_1 at and
    below theta_cs, to rounding level."""
    cb, sb = pp.cs_coefficients(family)
    th = oracle.cs_theta("double", family)
    for frac, idx in ((1.0, 0), (0.5, 1)):
        A = inputs.matrix(18, "normal", 1.0, index=150 + idx, sub=family)
        t = float(np.sqrt(frac * th / oracle.norm1(A)))
        C, S, _ = oracle.cs(A, t, family=family, sigma=0)
        B = t * t * A
        assert relfro(C, _horner(cb, B)) < 1e-14
        assert relfro(S, t * _horner(sb, B)) < 1e-14
