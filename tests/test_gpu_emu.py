"""The FP64 path with every product emulated on the BF16 tensor cores
("fp64_emu": eight 7-bit slices per row / column, 36 slice products).

One product is checked elementwise against the FP64 oracle product with the
bound |P - P_ref| <= 4 K u (|X| |Y|) + 2^-52 K max|X_i.| max|Y_.j|,
u = 2^-53: the oracle's own rounding plus the emulation's worst case (slice
residuals and dropped slice pairs), including rows and columns of very
different scales; small-integer operands must come out exact.  The whole
method is held to the FP64 path's bound against the oracle (1e-11)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2010_00465_gb300 import api, inputs

pytestmark = pytest.mark.gpu
U = 2.0 ** -53
TOL64 = 1e-11


def relfro(X, Y):
    X = np.asarray(X)
    Y = np.asarray(Y)
    return float(np.linalg.norm(X - Y) / max(np.linalg.norm(Y), 1e-300))


def dev(A):
    return torch.from_numpy(np.ascontiguousarray(A)).cuda()


def check_product(X, Y):
    P = api.matmul(dev(X), dev(Y), "fp64_emu").cpu().numpy()
    ref = oracle.matmul(X, Y)
    K = X.shape[1]
    rowmax = np.abs(X).max(axis=1, keepdims=True)
    colmax = np.abs(Y).max(axis=0, keepdims=True)
    bound = 4 * K * U * (np.abs(X) @ np.abs(Y)) + 2.0 ** -52 * K * rowmax * colmax
    assert np.all(np.abs(P - ref) <= bound + 1e-300), float(np.max(np.abs(P - ref) / (bound + 1e-300)))
    return P, ref


@pytest.mark.parametrize("n", [1, 2, 5, 31, 64, 127, 128, 129, 300, 513])
def test_product_bound(n):
    X = inputs.matrix(n, "normal", None, index=190, sub=n)
    Y = inputs.matrix(n, "uniform_pm", None, index=191, sub=n)
    P, ref = check_product(X, Y)
    assert relfro(P, ref) <= 1e-15


@pytest.mark.parametrize("n", [1152, 1300])
@pytest.mark.parametrize("slices", [8, 4])
def test_product_split_last_round(n, slices):
    """More tiles than a 152-SM GB300 runs at once and K over two 512-k chunks:
    the persistent grid's last, partial round runs as K halves on different
    CTAs (1152: 162 tiles, halves of one and two chunks; 1300: ragged edges)
    and must still meet the product's bound everywhere."""
    X = inputs.matrix(n, "normal", None, index=196, sub=n)
    Y = inputs.matrix(n, "normal", None, index=197, sub=n)
    if slices == 8:
        check_product(X, Y)
        return
    P = api.matmul(dev(X), dev(Y), "split_bf16").cpu().numpy()
    ref = oracle.matmul(X, Y)
    rowmax = np.abs(X).max(axis=1, keepdims=True)
    colmax = np.abs(Y).max(axis=0, keepdims=True)
    bound = 4 * n * U * (np.abs(X) @ np.abs(Y)) + 2.0 ** -25 * n * rowmax * colmax
    assert np.all(np.abs(P - ref) <= bound), float(np.max(np.abs(P - ref) / bound))


def test_product_long_k():
    """K = 1536 spans three promotion chunks of 512."""
    n = 1536
    X = inputs.matrix(n, "normal", None, index=192)
    Y = inputs.matrix(n, "normal", None, index=193)
    check_product(X, Y)


def test_product_row_and_column_scales():
    """Per-row and per-column exponents: rows and columns scaled by 2^-40 ..
    2^40, plus zero rows and columns."""
    n = 200
    g = inputs.rng(194)
    X = g.standard_normal((n, n)) * np.exp2(g.integers(-40, 41, size=(n, 1)))
    Y = g.standard_normal((n, n)) * np.exp2(g.integers(-40, 41, size=(1, n)))
    X[7] = 0.0
    Y[:, 11] = 0.0
    P, ref = check_product(X, Y)
    assert not P[7].any() and not P[:, 11].any()


def test_product_integer_exactness():
    """Small-integer operands have an exact product in FP64; the emulation
    must reproduce it bit for bit (every level sums exactly)."""
    n = 257
    g = inputs.rng(195)
    X = g.integers(-1000, 1001, size=(n, n)).astype(np.float64)
    Y = g.integers(-1000, 1001, size=(n, n)).astype(np.float64)
    P = api.matmul(dev(X), dev(Y), "fp64_emu").cpu().numpy()
    assert np.array_equal(P, X @ Y)


def _two_prod(a, b):
    """Exact product a b = p + e (Dekker's splitting, no FMA)."""
    c = 134217729.0
    t = c * a
    ah = t - (t - a)
    al = a - ah
    t = c * b
    bh = t - (t - b)
    bl = b - bh
    p = a * b
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def test_product_full_size_against_exact_rows():
    """n = 4096: sampled rows of X Y against the exactly rounded product
    (error-free products summed with math.fsum): the emulated product is at
    least as accurate as the native FP64 product."""
    n = 4096
    X = inputs.matrix(n, "normal", None, index=201)
    Y = inputs.matrix(n, "normal", None, index=202)
    Xd, Yd = dev(X), dev(Y)
    Pe = api.matmul(Xd, Yd, "fp64_emu").cpu().numpy()
    P64 = api.matmul(Xd, Yd, "fp64").cpu().numpy()
    rows = [0, 1777, 4095]
    ref = np.zeros((len(rows), n))
    for ii, i in enumerate(rows):
        p, e = _two_prod(X[i][:, None], Y)
        for j in range(n):
            ref[ii, j] = math.fsum(np.concatenate((p[:, j], e[:, j])))
    err_e = relfro(Pe[rows], ref)
    err_64 = relfro(P64[rows], ref)
    assert err_e <= 2e-15 and err_e <= err_64, (err_e, err_64)


@pytest.mark.parametrize("n", [1, 5, 64, 129, 200])
@pytest.mark.parametrize("nrm", [2.0 ** -6, 0.5, 2.0, 8.0, 64.0])
def test_cossin_matches_oracle(n, nrm):
    A = inputs.matrix(n, "normal", nrm, index=196, sub=n)
    Co, So, io = oracle.cossin(A)
    C, S, info = api.cossin(dev(A), "fp64_emu", return_info=True)
    assert (info["m"], info["s"], info["table"]) == (io["m"], io["s"], 0)
    assert relfro(C.cpu(), Co) <= TOL64
    assert relfro(S.cpu(), So) <= TOL64


@pytest.mark.parametrize("family", ["symmetric", "triangular", "nilpotent", "uniform01"])
@pytest.mark.parametrize("nrm", [1.0, 64.0])
def test_families(family, nrm):
    A = inputs.matrix(130, family, nrm, index=197)
    Co, So, _ = oracle.cossin(A)
    C, S = api.cossin(dev(A), "fp64_emu")
    assert relfro(C.cpu(), Co) <= TOL64 and relfro(S.cpu(), So) <= TOL64


@pytest.mark.parametrize("m", [4, 8, 9, 16, 24])
def test_every_family_forced(m):
    A = inputs.matrix(96, "normal", 1.0, index=198, sub=m)
    Co, So, _ = oracle.cossin(A, m=m, s=2)
    C, S = api.cossin(dev(A), "fp64_emu", m=m, s=2)
    assert relfro(C.cpu(), Co) <= TOL64 and relfro(S.cpu(), So) <= TOL64


@pytest.mark.parametrize("family,nrm", [("normal", 2.0 ** -4), ("normal", 1.0), ("normal", 8.0), ("normal", 64.0),
                                        ("symmetric", 8.0), ("triangular", 8.0)])
def test_full_size_against_fp64_path(family, nrm):
    """n = 4096 (the benchmark workload): against the native FP64 path.  The
    difference is the sum of both paths' rounding, and the native product's
    own (2e-15 per product at K = 4096 against an exact reference, above the
    emulation's; see test_product_full_size_against_exact_rows) grows about
    4-fold per double-angle step: 8e-12 at ||A||_1 = 64 (s = 6).  Bound
    1e-12 up to ||A||_1 = 8, 2e-11 at 64."""
    A = dev(inputs.matrix(4096, family, nrm, index=199))
    C64, S64, i64 = api.cossin(A, "fp64", return_info=True)
    C, S, info = api.cossin(A, "fp64_emu", return_info=True)
    assert (info["m"], info["s"]) == (i64["m"], i64["s"])
    tol = 1e-12 if nrm <= 8 else 2e-11
    assert float((C - C64).norm() / C64.norm()) <= tol
    assert float((S - S64).norm() / S64.norm()) <= tol


def test_cs_and_unitary_forms():
    A = inputs.matrix(100, "symmetric", 3.0, index=200)
    Co, So, io = oracle.cs(A, 1.3)
    C, S, info = api.cossin_cs(dev(A), 1.3, "fp64_emu", return_info=True)
    assert (info["m"], info["s"]) == (io["m"], io["s"])
    assert relfro(C.cpu(), Co) <= TOL64 and relfro(S.cpu(), So) <= TOL64
    Uo, _ = oracle.unitary(A, 0.8)
    Ug = api.unitary(dev(A), 0.8, "fp64_emu")
    assert relfro(Ug.cpu().numpy(), Uo) <= TOL64


@pytest.mark.parametrize("nrm", [1.0, 64.0])
def test_n8192_block_diagonal(nrm):
    """The largest order the emulated products accept (K = 8192): a permuted
    block-diagonal matrix, sampled 64-blocks against the oracle."""
    n, block = 8192, 64
    g = inputs.rng(203)
    perm = g.permutation(n)
    A = np.zeros((n, n))
    blocks = [inputs.matrix(block, "normal", nrm, index=203, sub=i) for i in range(n // block)]
    for i, B in enumerate(blocks):
        idx = perm[i * block:(i + 1) * block]
        A[np.ix_(idx, idx)] = B
    C, S, info = api.cossin(dev(A), "fp64_emu", return_info=True)
    assert (info["m"], info["s"]) == oracle.select(oracle.norm1(A), "double")
    C = C.cpu().numpy()
    S = S.cpu().numpy()
    for i in list(range(0, n // block, 29)) + [n // block - 1]:
        idx = perm[i * block:(i + 1) * block]
        Co, So, _ = oracle.cossin(A[np.ix_(idx, idx)], m=info["m"], s=info["s"])
        assert relfro(C[np.ix_(idx, idx)], Co) <= TOL64
        assert relfro(S[np.ix_(idx, idx)], So) <= TOL64
