"""Pins of the oracle's propagator exp(-i t A) = cos(tA) - i sin(tA) (Sec. 1)
and of its gradient, against eigendecompositions, scipy's expm on the complex
matrix, unitarity and finite differences -- nothing here uses the CUDA path."""
import numpy as np
import pytest

import oracle
from paper_2010_00465_gb300 import inputs


def relfro(X, Y):
    return float(np.linalg.norm(X - Y) / max(np.linalg.norm(Y), 1e-300))


@pytest.mark.parametrize("t", [0.05, 1.0, 7.5, -2.0])
def test_symmetric_is_unitary_and_matches_eigen(t):
    A = inputs.matrix(24, "symmetric", 4.0, index=170)
    U, info = oracle.unitary(A, t)
    lam, V = np.linalg.eigh(A)
    Ue = (V * np.exp(-1j * t * lam)) @ V.T
    tol = 1e-14 * (1 + 4.0 ** info["s"])
    assert np.abs(U - Ue).max() <= tol
    assert np.abs(U @ U.conj().T - np.eye(24)).max() <= tol


@pytest.mark.parametrize("family", ["normal", "triangular", "uniform_pm"])
@pytest.mark.parametrize("t", [0.3, 2.0])
def test_general_against_complex_expm(family, t):
    sl = pytest.importorskip("scipy.linalg")
    A = inputs.matrix(15, family, 3.0, index=171)
    U, _ = oracle.unitary(A, t)
    E = sl.expm(-1j * t * A)
    assert np.abs(U - E).max() <= 1e-12 * max(1.0, np.abs(E).max())


def test_zero_time_and_group_property():
    A = inputs.matrix(10, "symmetric", 2.0, index=172)
    U0, info = oracle.unitary(A, 0.0)
    assert np.array_equal(U0, np.eye(10)) and info["norm1"] == 0.0
    U1, _ = oracle.unitary(A, 0.4)
    U2, _ = oracle.unitary(A, 0.8)
    assert relfro(U2, U1 @ U1) < 1e-13


@pytest.mark.parametrize("t", [0.7, -1.3])
def test_gradient_against_central_differences(t):
    n = 9
    A = inputs.matrix(n, "normal", 2.0, index=173)
    g = inputs.rng(174)
    G = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    _, info = oracle.unitary(A, t)
    m, s = info["m"], info["s"]
    dA = oracle.unitary_gradient(A, t, G, m, s)

    def loss(X):
        U, _ = oracle.unitary(X, t, m=m, s=s)
        return float(np.real(np.sum(np.conj(G) * U)))

    for k in range(3):
        E = g.standard_normal((n, n))
        h = 1e-6
        fd = (loss(A + h * E) - loss(A - h * E)) / (2 * h)
        assert abs(fd - float(np.sum(dA * E))) <= 1e-7 * max(1.0, abs(fd)), k
