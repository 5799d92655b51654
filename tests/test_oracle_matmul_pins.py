"""Pins of the oracle's plain product (the reference of the product tests):
exact on integer operands, within the classical rounding bound of the exactly
rounded product (Higham, Accuracy and Stability of Numerical Algorithms,
Sec. 3.5: |fl(XY) - XY| <= gamma_K |X||Y|, gamma_K = K u / (1 - K u)), and
transpose-equivariant bit for bit (a fixed summation order without
contraction)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2010_00465_gb300 import inputs

U = 2.0 ** -53


@pytest.mark.parametrize("n", [1, 3, 17, 64])
def test_integer_operands_are_exact(n):
    g = inputs.rng(300, n)
    X = g.integers(-2 ** 20, 2 ** 20, size=(n, n))
    Y = g.integers(-2 ** 20, 2 ** 20, size=(n, n))
    Z = oracle.matmul(X.astype(np.float64), Y.astype(np.float64))
    assert np.array_equal(Z, (X @ Y).astype(np.float64))  # |entries| < 2^47: exact in both


@pytest.mark.parametrize("n", [5, 24])
def test_within_the_rounding_bound_of_the_exact_product(n):
    X = inputs.matrix(n, "normal", None, index=301, sub=n)
    Y = inputs.matrix(n, "uniform_pm", None, index=302, sub=n)
    Z = oracle.matmul(X, Y)
    gamma = n * U / (1 - n * U)
    absXY = np.abs(X) @ np.abs(Y)
    for i in range(n):
        for j in range(n):
            exact = sum((Fraction(X[i, k]) * Fraction(Y[k, j]) for k in range(n)), Fraction(0))
            assert abs(Fraction(Z[i, j]) - exact) <= Fraction(gamma * absXY[i, j]) * (1 + Fraction(1, 10 ** 6))


def test_transpose_equivariance_is_bitwise():
    X = inputs.matrix(37, "normal", None, index=303)
    Y = inputs.matrix(37, "symmetric", None, index=304) + inputs.matrix(37, "normal", None, index=305)
    assert np.array_equal(oracle.matmul(X, Y).T, oracle.matmul(Y.T.copy(), X.T.copy()))


def test_identity_and_zero():
    X = inputs.matrix(20, "normal", None, index=306)
    assert np.array_equal(oracle.matmul(X, np.eye(20)), X)
    assert np.array_equal(oracle.matmul(np.eye(20), X), X)
    assert not oracle.matmul(X, np.zeros((20, 20))).any()
