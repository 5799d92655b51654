"""Pins of the FP64 oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself or with the CUDA path.  Each
test would fail on a plausible slip in ``oracle/cossin_oracle.c``: a dropped
term or wrong sign in a scheme (Taylor coefficients read off a nilpotent shift
matrix), a mistyped coefficient (comparison with the high-precision expansion
of the printed coefficients), a wrong theta entry (Tables 1-2 and their
recomputation from the Sec. 3 error series), a wrong double-angle step
(closed forms and identities at s > 0), a transposed operand (non-symmetric
closed forms, brute-force series).
"""
import math

import mpmath as mp
import numpy as np
import pytest

import oracle
import paper_poly as pp
from paper_2010_00465_gb300 import inputs

FAM = {4: ("c4", "s5", 4, 5), 8: ("c8", "s79", 8, 7), 9: ("c8", "s9", 8, 9), 16: ("c16", "s17", 16, 17),
       24: ("c24", "s23", 24, 21)}
U = {"double": 2.0 ** -53, "single": 2.0 ** -24}


def relfro(X, Y):
    return float(np.linalg.norm(X - Y) / max(np.linalg.norm(Y), 1e-300))


def shift(d):
    return np.diag(np.ones(d - 1), 1)


# ---------------------------------------------------------------- tables ---

def test_theta_table_is_the_papers():
    T = pp.tables()
    for prec in ("double", "single"):
        for i, m in enumerate((4, 8, 16, 24)):
            assert oracle.theta(prec, m, False) == T["theta"][prec]["cos"][i]
            want = T["theta"][prec]["sin"][i]
            if prec == "double" and m == 24:
                want = T["theta_reading"]["double"]["sin24"]
            assert oracle.theta(prec, m, True) == want


@pytest.mark.slow
def test_theta_recomputed_from_error_series():
    """Sec. 3: theta_2m is the largest ||A|| whose error bound (150 terms) is <= u.
    Recomputed from the printed coefficients (k = 7 polished by Newton) it must
    agree with the oracle's table to the printed digits."""
    polys = pp.schemes(refined=True)
    for prec in ("double", "single"):
        for m, (ck, sk, _, _) in FAM.items():
            if m == 9:
                continue  # no table entry; see test_t9_sine_variant
            for key, sine in ((ck, False), (sk, True)):
                th = float(pp.theta(polys[key], sine, mp.mpf(2) ** (-53 if prec == "double" else -24)))
                got = oracle.theta(prec, m, sine)
                assert abs(th - got) <= 6e-5 * got, (prec, key, th, got)


def test_paper_sin24_double_entry_is_not_reproduced():
    """The one deliberate deviation from Table 1 (documented reading)."""
    polys = pp.schemes(refined=True)
    th = float(pp.theta(polys["s23"], True, mp.mpf(2) ** -53))
    assert abs(th - 1.8555) < 1e-4
    assert abs(th - pp.tables()["theta"]["double"]["sin"][3]) > 0.1


def test_printed_coefficients_match_taylor():
    """Sec. 2.1: each scheme reproduces the Taylor series through its order
    (the k = 7 sine only through A^21, see the theta reading)."""
    polys = pp.schemes(refined=False)
    for m, (ck, sk, oc, os_) in FAM.items():
        for k in range(oc + 1):
            assert abs(polys[ck][k] - pp.cos_taylor(k)) < mp.mpf(10) ** -19, (ck, k)
        for k in range(os_ + 1):
            assert abs(polys[sk][k] - pp.sin_taylor(k)) < mp.mpf(10) ** -18 * max(1, abs(pp.sin_taylor(k)) * 1e3), (sk, k)
    # the k = 7 sine misses A^23 by a relative -1.785
    a23 = (polys["s23"][23] - pp.sin_taylor(23)) / pp.sin_taylor(23)
    assert abs(float(a23) + 1.785) < 1e-3


def test_selection_on_workload_norms():
    """(2m, s) for the norms of the n = 4096 and 64 x 64 workloads, derived by
    hand from Tables 1-2 with the minimal-cost reading."""
    want = {
        "double": {2.0 ** -4: (8, 0), 1.0: (24, 0), 8.0: (24, 3), 64.0: (24, 6), 2.0: (24, 1)},
        "single": {2.0 ** -4: (4, 0), 1.0: (16, 0), 8.0: (24, 1), 64.0: (24, 4), 16.0: (24, 2)},
    }
    for prec, table in want.items():
        for nrm, ms in table.items():
            assert oracle.select(nrm, prec) == ms, (prec, nrm)


def test_selection_is_cost_minimal_and_admissible():
    T = pp.tables()
    pis = dict(zip(T["products"]["2m"], T["products"]["Pi"]))
    for prec in ("double", "single"):
        th = {m: min(oracle.theta(prec, m, False), oracle.theta(prec, m, True)) for m in (4, 8, 16, 24)}
        for nrm in np.geomspace(1e-6, 1e6, 301):
            m, s = oracle.select(nrm, prec)
            assert nrm / 2.0 ** s <= th[m]
            assert s == 0 or nrm / 2.0 ** (s - 1) > th[m]
            cost = pis[m] + 2 * s
            for m2 in (4, 8, 16, 24):
                s2 = max(0, math.ceil(math.log2(nrm / th[m2]))) if nrm > th[m2] else 0
                while nrm / 2.0 ** s2 > th[m2]:
                    s2 += 1
                assert cost <= pis[m2] + 2 * s2


def test_selection_edge_cases():
    assert oracle.select(0.0, "double") == (4, 0)
    with pytest.raises(oracle.OracleError):
        oracle.select(float("inf"), "double")
    with pytest.raises(oracle.OracleError):
        oracle.select(float("nan"), "single")
    with pytest.raises(oracle.OracleError):
        oracle.select(1e300, "double")  # would need s > 64


def test_norm1_definition():
    A = inputs.matrix(37, "normal", index=11)
    assert oracle.norm1(A) == float(np.abs(A).sum(axis=0).max())
    assert oracle.norm1(np.zeros((0, 0))) == 0.0
    B = A.copy()
    B[3, 5] = np.nan
    assert math.isnan(oracle.norm1(B))


# ------------------------------------------------- scheme coefficients ---

@pytest.mark.parametrize("m", [4, 8, 9, 16, 24])
def test_chain_coefficients_on_nilpotent_shift(m):
    """For the shift matrix N (N^k has ones on the k-th superdiagonal and
    N^d = 0), p(N) has the coefficient of A^k of the approximant p in entry
    (0, k).  The oracle's chain, read this way, must equal the Taylor series
    through the scheme's order and the high-precision expansion of the printed
    coefficients at every power."""
    ck, sk, oc, os_ = FAM[m]
    polys = pp.schemes(refined=False)
    d = len(polys[sk]) + 1
    C, S, info = oracle.cossin(shift(d), "double", m=m, s=0)
    assert (info["m"], info["s"]) == (m, 0)
    for k in range(d):
        ref_c = float(polys[ck][k]) if k < len(polys[ck]) else 0.0
        ref_s = float(polys[sk][k]) if k < len(polys[sk]) else 0.0
        assert C[0, k] == pytest.approx(ref_c, rel=1e-13, abs=1e-300), ("cos", k)
        assert S[0, k] == pytest.approx(ref_s, rel=1e-13, abs=1e-300), ("sin", k)
    for k in range(oc + 1):
        assert C[0, k] == pytest.approx(float(pp.cos_taylor(k)), rel=1e-14, abs=0), ("cos taylor", k)
    for k in range(os_ + 1):
        assert S[0, k] == pytest.approx(float(pp.sin_taylor(k)), rel=1e-14, abs=0), ("sin taylor", k)
    # A nilpotent matrix has a terminating series: every row of p(N) repeats the pattern.
    assert np.allclose(np.triu(C, 0)[1, 1:], C[0, :-1], rtol=1e-14, atol=0)


@pytest.mark.parametrize("m,s", [(24, 3), (16, 2), (8, 1), (9, 2), (4, 2)])
def test_double_angle_on_nilpotent_shift(m, s):
    """With s double-angle steps on A_s = 2^-s A, the composite approximant
    still matches the Taylor series of cos A and sin A through the family's
    order (Sec. 1: cos 2X = 2cos^2 X - I, sin 2X = 2 sin X cos X)."""
    ck, sk, oc, os_ = FAM[m]
    d = 30
    C, S, _ = oracle.cossin(shift(d), "double", m=m, s=s)
    for k in range(min(oc, d - 1) + 1):
        assert C[0, k] == pytest.approx(float(pp.cos_taylor(k)), rel=1e-13, abs=1e-300), k
    for k in range(min(os_, d - 1) + 1):
        assert S[0, k] == pytest.approx(float(pp.sin_taylor(k)), rel=1e-13, abs=1e-300), k


# ------------------------------------------------------- closed forms ---

@pytest.mark.parametrize("nrm", [2.0 ** -6, 2.0 ** -4, 0.5, 1.0, 3.0, 8.0, 64.0])
def test_diagonal(nrm):
    g = inputs.rng(21, int(nrm * 64))
    d = g.uniform(-1, 1, size=17)
    d *= nrm / np.abs(d).max()
    C, S, info = oracle.cossin(np.diag(d))
    # rounding of size u grows by at most about a factor 2 per double-angle step
    tol = 2e-15 * 2.0 ** info["s"] + 1e-14
    assert relfro(C, np.diag(np.cos(d))) < tol
    assert relfro(S, np.diag(np.sin(d))) < tol


@pytest.mark.parametrize("nrm", [2.0 ** -4, 1.0, 8.0, 64.0])
def test_symmetric_via_eigendecomposition(nrm):
    A = inputs.matrix(24, "symmetric", nrm, index=22)
    w, V = np.linalg.eigh(A)
    C, S, _ = oracle.cossin(A)
    tol = 1e-13 * max(1.0, nrm / 8)
    assert relfro(C, (V * np.cos(w)) @ V.T) < tol
    assert relfro(S, (V * np.sin(w)) @ V.T) < tol


@pytest.mark.parametrize("t", [0.05, 0.7, 1.5, 3.0, 10.0])
def test_rotation_generator(t):
    """K = [[0,1],[-1,0]] has K^2 = -I, so cos(tK) = cosh(t) I, sin(tK) = sinh(t) K;
    J = [[0,1],[1,0]] has J^2 = I, so cos(tJ) = cos(t) I, sin(tJ) = sin(t) J."""
    K = np.array([[0.0, 1.0], [-1.0, 0.0]])
    J = np.array([[0.0, 1.0], [1.0, 0.0]])
    C, S, _ = oracle.cossin(t * K)
    assert relfro(C, math.cosh(t) * np.eye(2)) < 1e-14
    assert relfro(S, math.sinh(t) * K) < 1e-14
    C, S, _ = oracle.cossin(t * J)
    assert np.abs(C - math.cos(t) * np.eye(2)).max() < 1e-14 * max(1, t)
    assert np.abs(S - math.sin(t) * J).max() < 1e-14 * max(1, t)


@pytest.mark.parametrize("lam_exp", range(0, 9))
@pytest.mark.parametrize("target", [0.1, 2.0, 64.0])
def test_jordan2_family(lam_exp, target):
    """Sec. 4 family A = [[1, lam], [0, -1]]: A^2 = I, so for X = alpha A,
    cos X = cos(alpha) I and sin X = sin(alpha) A.  Large lam overscales."""
    A = inputs.jordan2(10.0 ** lam_exp)
    alpha = target / np.abs(A).sum(axis=0).max()
    C, S, info = oracle.cossin(alpha * A)
    # s double-angle steps amplify a rounding error of size u*||X|| by about 2^s
    tol = 1e-15 * (1 + 4.0 ** info["s"]) * max(1.0, 10.0 ** lam_exp * alpha)
    assert np.abs(C - math.cos(alpha) * np.eye(2)).max() <= tol + 1e-15
    assert np.abs(S - math.sin(alpha) * A).max() <= tol * max(1.0, 10.0 ** lam_exp) + 1e-15


@pytest.mark.parametrize("n", [2, 5, 8, 13])
def test_nilpotent_terminates(n):
    """Strictly upper triangular A: A^n = 0, so cos and sin are finite sums."""
    A = inputs.matrix(n, "nilpotent", 3.0, index=23, sub=n)
    C, S, _ = oracle.cossin(A)
    P = np.eye(n)
    Cref = np.zeros((n, n))
    Sref = np.zeros((n, n))
    for k in range(n):
        if k % 2 == 0:
            Cref += (-1) ** (k // 2) / math.factorial(k) * P
        else:
            Sref += (-1) ** ((k - 1) // 2) / math.factorial(k) * P
        P = P @ A
    assert relfro(C, Cref) < 1e-14
    assert relfro(S, Sref) < 1e-14


# ---------------------------------------------------------- identities ---

@pytest.mark.parametrize("family", ["normal", "uniform01", "uniform_pm", "triangular"])
@pytest.mark.parametrize("nrm", [0.3, 2.0, 8.0, 64.0])
def test_pythagoras(family, nrm):
    A = inputs.matrix(20, family, nrm, index=24)
    C, S, _ = oracle.cossin(A)
    R = C @ C + S @ S - np.eye(20)
    scale = max(1.0, np.linalg.norm(C @ C) + np.linalg.norm(S @ S))
    assert np.linalg.norm(R) / scale < 1e-12


@pytest.mark.parametrize("nrm", [0.5, 2.0, 8.0])
def test_double_angle_identity(nrm):
    A = inputs.matrix(16, "normal", nrm, index=25)
    C, S, _ = oracle.cossin(A)
    C2, S2, _ = oracle.cossin(2 * A)
    assert relfro(C2, 2 * C @ C - np.eye(16)) < 1e-12
    assert relfro(C2, np.eye(16) - 2 * S @ S) < 1e-12
    assert relfro(S2, 2 * S @ C) < 1e-12


def test_commute_with_A():
    A = inputs.matrix(12, "normal", 5.0, index=26)
    C, S, _ = oracle.cossin(A)
    assert np.linalg.norm(C @ A - A @ C) < 1e-12 * np.linalg.norm(A) * np.linalg.norm(C)
    assert np.linalg.norm(S @ A - A @ S) < 1e-12 * np.linalg.norm(A) * np.linalg.norm(S)


def test_zero_and_empty():
    C, S, info = oracle.cossin(np.zeros((5, 5)))
    assert np.array_equal(C, np.eye(5)) and np.array_equal(S, np.zeros((5, 5)))
    C, S, info = oracle.cossin(np.zeros((0, 0)))
    assert C.shape == (0, 0)


def test_transpose_equivariance():
    """f(A^T) = f(A)^T for a polynomial; catches a transposed operand."""
    A = inputs.matrix(15, "triangular", 4.0, index=27)
    C, S, _ = oracle.cossin(A)
    Ct, St, _ = oracle.cossin(A.T.copy())
    assert relfro(Ct, C.T) < 1e-14 and relfro(St, S.T) < 1e-14


# ------------------------------------------------------- brute force ---

def _mp_series(A, terms=160):
    n = A.shape[0]
    M = mp.matrix(A.tolist())
    P = mp.eye(n)
    Cs = mp.zeros(n, n)
    Ss = mp.zeros(n, n)
    for k in range(terms):
        if k % 2 == 0:
            Cs += P * (mp.mpf(-1) ** (k // 2) / mp.factorial(k))
        else:
            Ss += P * (mp.mpf(-1) ** ((k - 1) // 2) / mp.factorial(k))
        P = P * M
    f = lambda X: np.array([[float(X[i, j]) for j in range(n)] for i in range(n)])
    return f(Cs), f(Ss)


@pytest.mark.parametrize("family", ["normal", "uniform01", "triangular", "symmetric"])
@pytest.mark.parametrize("nrm", [0.05, 1.0, 4.0, 8.0])
def test_brute_force_series(family, nrm):
    """A 60-digit Taylor series with 160 terms stands in for the 100-digit
    reference solutions of Sec. 4."""
    mp.mp.dps = 60
    A = inputs.matrix(6, family, nrm, index=28)
    Cr, Sr = _mp_series(A)
    C, S, _ = oracle.cossin(A)
    assert relfro(C, Cr) < 1e-13
    assert relfro(S, Sr) < 1e-13


def test_single_table_accuracy():
    """With the single table the truncation error is bounded by about 2^-24."""
    mp.mp.dps = 60
    for nrm in (0.1, 1.0, 4.0, 30.0):
        A = inputs.matrix(6, "normal", nrm, index=29)
        Cr, Sr = _mp_series(A, terms=200)
        C, S, info = oracle.cossin(A, "single")
        assert relfro(C, Cr) < 5e-7 * 2 ** info["s"]
        assert relfro(S, Sr) < 5e-7 * 2 ** info["s"]


@pytest.mark.parametrize("m", [4, 8, 16, 24])
@pytest.mark.parametrize("prec", ["double", "single"])
def test_truncation_bound_at_theta(m, prec):
    """Sec. 3: at ||A|| = theta_2m (s = 0) the forward error is at most u.
    For a 1 x 1 matrix [x], x > 0, the bound is attained up to sign pattern."""
    th = min(oracle.theta(prec, m, False), oracle.theta(prec, m, True))
    mp.mp.dps = 40
    for x in (th, 0.5 * th):
        C, S, _ = oracle.cossin(np.array([[x]]), prec, m=m, s=0)
        ec = abs(C[0, 0] - float(mp.cos(x)))
        es = abs(S[0, 0] - float(mp.sin(x)))
        assert ec <= U[prec] + 4 * 2.0 ** -53, (m, x, ec)
        assert es <= U[prec] + 4 * 2.0 ** -53 * max(1, x), (m, x, es)


@pytest.mark.parametrize("prec", ["double", "single"])
def test_t9_sine_variant(prec):
    """2m = 9: T8c with the five-product sine T9s (eq. Algorithm5sA).  Its
    sine's admissible norm, recomputed from the Sec. 3 series (the paper
    prints none), is 0.17402 (double) / 1.0813 (single), above the cosine's
    Table value, so the pair is bound by theta^c_8; at that norm the forward
    error of both is at most u, and the sine error stays at most u up to its
    own theta.  It costs 5 products."""
    polys = pp.schemes()
    th_s = float(pp.theta(polys["s9"], True, U[prec]))
    assert th_s == pytest.approx({"double": 0.17402, "single": 1.0813}[prec], rel=2e-4)
    th = min(oracle.theta(prec, 8, False), th_s)
    assert th == oracle.theta(prec, 8, False)
    mp.mp.dps = 40
    for x in (th, 0.5 * th):
        C, S, info = oracle.cossin(np.array([[x]]), prec, m=9, s=0)
        assert info["products"] == 5
        assert abs(C[0, 0] - float(mp.cos(x))) <= U[prec] + 4 * 2.0 ** -53
        assert abs(S[0, 0] - float(mp.sin(x))) <= U[prec] + 4 * 2.0 ** -53
    C, S, _ = oracle.cossin(np.array([[th_s]]), prec, m=9, s=0)
    assert abs(S[0, 0] - float(mp.sin(th_s))) <= U[prec] + 4 * 2.0 ** -53
    # the T_{7,9} sine of 2m = 8 is above u there
    _, S8, _ = oracle.cossin(np.array([[th_s]]), prec, m=8, s=0)
    assert abs(S8[0, 0] - float(mp.sin(th_s))) > 2 * U[prec]


def test_scipy_library_routine():
    sl = pytest.importorskip("scipy.linalg")
    for nrm in (0.01, 1.0, 8.0, 64.0):
        A = inputs.matrix(30, "normal", nrm, index=30)
        C, S, _ = oracle.cossin(A)
        assert relfro(C, sl.cosm(A)) < 1e-12 * max(1, nrm / 8)
        assert relfro(S, sl.sinm(A)) < 1e-12 * max(1, nrm / 8)


# ------------------------------------------------------------ Frechet ---

def test_frechet_block_is_linear_and_matches_differences():
    A = inputs.matrix(7, "normal", 3.0, index=31)
    E = inputs.matrix(7, "normal", 1.0, index=32)
    m, s = oracle.select(oracle.norm1(A), "double")
    Lc, Ls = oracle.frechet(A, E, m, s)
    Lc2, Ls2 = oracle.frechet(A, 2.5 * E, m, s)
    assert relfro(Lc2, 2.5 * Lc) < 1e-13 and relfro(Ls2, 2.5 * Ls) < 1e-13
    h = 1e-5
    Cp, Sp, _ = oracle.cossin(A + h * E, m=m, s=s)
    Cm, Sm, _ = oracle.cossin(A - h * E, m=m, s=s)
    assert relfro((Cp - Cm) / (2 * h), Lc) < 1e-8
    assert relfro((Sp - Sm) / (2 * h), Ls) < 1e-8


def test_frechet_exact_for_commuting_direction():
    """For E = A the derivative of cos along A is -sin(A) A (scalar calculus)."""
    A = inputs.matrix(6, "symmetric", 2.0, index=33)
    m, s = oracle.select(oracle.norm1(A), "double")
    Lc, Ls = oracle.frechet(A, A, m, s)
    C, S, _ = oracle.cossin(A)
    assert relfro(Lc, -S @ A) < 1e-12
    assert relfro(Ls, C @ A) < 1e-12


def test_gradient_adjoint_identity():
    """<G, L(A, E)> = <L(A^T, G), E> for every E (real polynomial)."""
    A = inputs.matrix(6, "triangular", 5.0, index=34)
    G = inputs.matrix(6, "normal", None, index=35)
    E = inputs.matrix(6, "normal", None, index=36)
    m, s = oracle.select(oracle.norm1(A), "double")
    Lc, Ls = oracle.frechet(A, E, m, s)
    gc = oracle.gradient(A, G, np.zeros_like(G), m, s)
    gs = oracle.gradient(A, np.zeros_like(G), G, m, s)
    assert abs(np.sum(G * Lc) - np.sum(gc * E)) < 1e-11 * np.abs(G).sum() * np.abs(Lc).max()
    assert abs(np.sum(G * Ls) - np.sum(gs * E)) < 1e-11 * np.abs(G).sum() * np.abs(Ls).max()


def _horner(coef, A):
    """p(A) = sum_k coef[k] A^k by Horner's rule in FP64 (numpy products)."""
    n = A.shape[0]
    P = float(coef[-1]) * np.eye(n)
    for c in reversed(coef[:-1]):
        P = P @ A + float(c) * np.eye(n)
    return P


@pytest.mark.parametrize("m", [4, 8, 9, 16, 24])
@pytest.mark.parametrize("family", ["normal", "symmetric", "triangular"])
def test_chain_equals_expanded_polynomial(m, family):
    """The factorised chain of each family equals its expanded polynomial
    (coefficients from the high-precision expansion of the printed ones)
    evaluated by Horner's rule, on random A at and below the family's
    admissible norm (s = 0), to rounding level."""
    ck, sk, _, _ = FAM[m]
    polys = pp.schemes(refined=False)
    mm = 8 if m == 9 else m
    th = min(oracle.theta("double", mm, False), oracle.theta("double", mm, True))
    for frac, idx in ((1.0, 0), (0.5, 1)):
        A = inputs.matrix(20, family, frac * th, index=140 + idx, sub=m)
        C, S, _ = oracle.cossin(A, "double", m=m, s=0)
        Ch = _horner(polys[ck], A)
        Sh = _horner(polys[sk], A)
        assert relfro(C, Ch) < 1e-14, (m, family, frac, relfro(C, Ch))
        assert relfro(S, Sh) < 1e-14, (m, family, frac, relfro(S, Sh))
