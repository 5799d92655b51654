"""The split-precision form on the BF16 tensor cores ("split_bf16").

Its Taylor-chain products are BF16 multi-term products of four 7-bit slices
per row of X and column of Y (29 bits of each row / column maximum, the 10
slice products with p + q <= 3, every level summed exactly); its double-angle
steps are the eight-slice products of "fp64_emu".

One four-slice product is checked elementwise against the FP64 oracle
product.  Per k the slices leave residuals of at most 2^-28 max|X_i.| max|Y_.j|
on each side and the dropped pairs (p + q >= 4, both >= 1) at most
4 2^-28 max|X_i.| max|Y_.j|, so |P - P_ref| <= 2^-25 K max|X_i.| max|Y_.j|
plus the oracle's own rounding; the test allows 2^-24 K.  Operands whose
entries need at most 29 bits below their row / column maximum (integers up to
2^10 here) come out exact.  The whole method is held to the bounds of the
other single-table forms against the oracle at the same (2m, s)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2010_00465_gb300 import api, inputs

pytestmark = pytest.mark.gpu
U = 2.0 ** -53
TOL32 = 2e-5


def relfro(X, Y):
    X = np.asarray(X)
    Y = np.asarray(Y)
    return float(np.linalg.norm(X - Y) / max(np.linalg.norm(Y), 1e-300))


def dev(A):
    return torch.from_numpy(np.ascontiguousarray(A)).cuda()


def check_product(X, Y):
    P = api.matmul(dev(X), dev(Y), "split_bf16").cpu().numpy()
    ref = oracle.matmul(X, Y)
    K = X.shape[1]
    rowmax = np.abs(X).max(axis=1, keepdims=True)
    colmax = np.abs(Y).max(axis=0, keepdims=True)
    bound = 4 * K * U * (np.abs(X) @ np.abs(Y)) + 2.0 ** -24 * K * rowmax * colmax
    assert np.all(np.abs(P - ref) <= bound + 1e-300), float(np.max(np.abs(P - ref) / (bound + 1e-300)))
    return P, ref


@pytest.mark.parametrize("n", [1, 2, 5, 31, 64, 127, 128, 129, 300, 513])
def test_product_bound(n):
    X = inputs.matrix(n, "normal", None, index=210, sub=n)
    Y = inputs.matrix(n, "uniform_pm", None, index=211, sub=n)
    P, ref = check_product(X, Y)
    assert relfro(P, ref) <= 1e-7


def test_product_long_k():
    """K = 1536 spans three 512-k accumulator chunks."""
    n = 1536
    X = inputs.matrix(n, "normal", None, index=212)
    Y = inputs.matrix(n, "normal", None, index=213)
    check_product(X, Y)


def test_product_row_and_column_scales():
    """Per-row and per-column exponents 2^-40 .. 2^40, zero rows and columns."""
    n = 200
    g = inputs.rng(214)
    X = g.standard_normal((n, n)) * np.exp2(g.integers(-40, 41, size=(n, 1)))
    Y = g.standard_normal((n, n)) * np.exp2(g.integers(-40, 41, size=(1, n)))
    X[3] = 0.0
    Y[:, 17] = 0.0
    P, _ = check_product(X, Y)
    assert not P[3].any() and not P[:, 17].any()


def test_product_integer_exactness():
    """Integers of at most 11 bits are cut exactly into four slices and every
    level sums exactly, so the product is exact."""
    n = 257
    g = inputs.rng(215)
    X = g.integers(-1000, 1001, size=(n, n)).astype(np.float64)
    Y = g.integers(-1000, 1001, size=(n, n)).astype(np.float64)
    P = api.matmul(dev(X), dev(Y), "split_bf16").cpu().numpy()
    assert np.array_equal(P, X @ Y)


def test_product_diagonal_is_exact():
    """X = I + E with tiny E: the diagonal goes through FP64, so the product
    keeps E's contribution to FP32-class accuracy relative to E, not to 1."""
    n = 256
    E = 1e-6 * inputs.matrix(n, "normal", None, index=216)
    X = np.eye(n) + E
    Y = np.eye(n) + E.T
    P = api.matmul(dev(X), dev(Y), "split_bf16").cpu().numpy()
    ref = oracle.matmul(X, Y)
    D = ref - np.eye(n)
    assert relfro(P - np.eye(n), D) <= 1e-6


@pytest.mark.parametrize("n", [1, 5, 64, 129, 200])
@pytest.mark.parametrize("nrm", [2.0 ** -6, 0.5, 2.0, 8.0, 64.0])
def test_cs_and_unitary_forms(n, nrm):
    A = inputs.matrix(n, "symmetric", nrm, index=217, sub=n)
    t = 1.3
    Co, So, io = oracle.cs(A, t, prec="single")
    C, S, info = api.cossin_cs(dev(A), t, "split_bf16", return_info=True)
    assert (info["m"], info["s"], info["table"]) == (io["m"], io["s"], 1)
    assert relfro(C.cpu(), Co) <= TOL32 and relfro(S.cpu(), So) <= TOL32
    Uo, _ = oracle.unitary(A, 0.8, prec="single")
    Ug = api.unitary(dev(A), 0.8, "split_bf16")
    assert relfro(Ug.cpu().numpy(), Uo) <= TOL32
