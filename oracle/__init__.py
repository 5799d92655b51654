"""FP64 CPU oracle for simultaneous matrix cos/sin -- TEST INFRASTRUCTURE ONLY.

A thin ctypes wrapper over ``cossin_oracle.c``, a plain restatement of the
method of arXiv:2010.00465 (Sec. 2.1 factorised Taylor schemes, Sec. 3 error
bounds / Tables 1-2, Sec. 1 double-angle recovery).  Only ``tests/``, the
smoke check and the benchmark's CPU-baseline leg may import this package; the
CUDA library never does, and this package never imports the library.

Every function here is pinned by tests that do not rely on it; see
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cossin_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

PREC = {"double": 0, "single": 1}


class OracleError(RuntimeError):
    pass


class _Info(ctypes.Structure):
    _fields_ = [("norm1", ctypes.c_double), ("m", ctypes.c_int), ("s", ctypes.c_int),
                ("products", ctypes.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_norm1.restype = ctypes.c_double
            lib.oracle_norm1.argtypes = [dp, ctypes.c_long]
            lib.oracle_theta.restype = ctypes.c_double
            lib.oracle_theta.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.oracle_select.restype = ctypes.c_int
            lib.oracle_select.argtypes = [ctypes.c_double, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
            lib.oracle_cossin.restype = ctypes.c_int
            lib.oracle_cossin.argtypes = [dp, ctypes.c_long, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, dp, dp, ctypes.POINTER(_Info)]
            lib.oracle_cs.restype = ctypes.c_int
            lib.oracle_cs.argtypes = [dp, ctypes.c_long, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, dp, dp, ctypes.POINTER(_Info)]
            lib.oracle_cs_theta.restype = ctypes.c_double
            lib.oracle_cs_theta.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.oracle_cs_select.restype = ctypes.c_int
            lib.oracle_cs_select.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_int)]
            lib.oracle_matmul.restype = None
            lib.oracle_matmul.argtypes = [dp, dp, dp, ctypes.c_long]
            lib.oracle_set_threads.restype = None
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_get_threads.restype = ctypes.c_int
            lib.oracle_get_threads.argtypes = []
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("expected a square matrix, got shape %r" % (a.shape,))
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(t: int) -> None:
    _load().oracle_set_threads(int(t))


def threads() -> int:
    return int(_load().oracle_get_threads())


def norm1(A) -> float:
    """Exact matrix 1-norm (Sec. 4: the 1-norm drives the algorithm)."""
    A = _f64(A)
    return float(_load().oracle_norm1(_ptr(A), A.shape[0]))


def theta(prec: str, m: int, sine: bool) -> float:
    """theta_2m from Table 1 (double) / Table 2 (single), as held by the oracle."""
    f = {4: 0, 8: 1, 16: 2, 24: 3}[m]
    return float(_load().oracle_theta(PREC[prec], f, int(bool(sine))))


def select(norm: float, prec: str = "double"):
    """(2m, s) chosen by the oracle's cost rule over Tables 1-2."""
    m = ctypes.c_int()
    s = ctypes.c_int()
    rc = _load().oracle_select(float(norm), PREC[prec], ctypes.byref(m), ctypes.byref(s))
    if rc != 0:
        raise OracleError("oracle_select failed with status %d" % rc)
    return m.value, s.value


def cossin(A, prec: str = "double", m: int | None = None, s: int | None = None):
    """Return (cos(A), sin(A), info) in FP64.

    ``m``/``s`` force the family 2m and the number of double-angle steps;
    both or neither must be given.  ``m = 9`` is the 2m = 8 cosine with the
    five-product T9 sine of eq. Algorithm5sA.
    """
    A = _f64(A)
    n = A.shape[0]
    C = np.zeros((n, n), dtype=np.float64)
    S = np.zeros((n, n), dtype=np.float64)
    info = _Info()
    fm = -1 if m is None else int(m)
    fs = -1 if s is None else int(s)
    rc = _load().oracle_cossin(_ptr(A), n, PREC[prec], fm, fs, _ptr(C), _ptr(S),
                               ctypes.byref(info))
    if rc != 0:
        raise OracleError("oracle_cossin failed with status %d" % rc)
    return C, S, {"norm1": info.norm1, "m": info.m, "s": info.s, "products": info.products}


CS_FAMILIES = {0: "k=3, P_{3,4}^s (2 products)", 1: "k=3, P_4^s (3 products)", 2: "k=4 (4 products)",
               3: "k=5 (5 products)"}


def cs(A, t: float, prec: str = "double", family: int | None = None, sigma: int | None = None):
    """(c(t^2 A), s(t, A), info) of Sec. 2.2: cos(sqrt(t^2 A)) and
    A^(-1/2) sin(sqrt(t^2 A)).  info["m"] is the family index 0..3 and
    info["s"] the number of double-angle steps sigma; info["norm1"] is ||t^2 A||_1."""
    A = _f64(A)
    n = A.shape[0]
    C = np.zeros((n, n), dtype=np.float64)
    S = np.zeros((n, n), dtype=np.float64)
    info = _Info()
    ff = -1 if family is None else int(family)
    fs = -1 if sigma is None else int(sigma)
    rc = _load().oracle_cs(_ptr(A), n, float(t), PREC[prec], ff, fs, _ptr(C), _ptr(S), ctypes.byref(info))
    if rc != 0:
        raise OracleError("oracle_cs failed with status %d" % rc)
    return C, S, {"norm1": info.norm1, "m": info.m, "s": info.s, "products": info.products}


def cs_theta(prec: str, family: int) -> float:
    return float(_load().oracle_cs_theta(PREC[prec], int(family)))


def cs_select(normB: float, prec: str = "double"):
    f = ctypes.c_int()
    s = ctypes.c_int()
    rc = _load().oracle_cs_select(float(normB), PREC[prec], ctypes.byref(f), ctypes.byref(s))
    if rc != 0:
        raise OracleError("oracle_cs_select failed with status %d" % rc)
    return f.value, s.value


def unitary(A, t: float, prec: str = "double", m: int | None = None, s: int | None = None):
    """U = exp(-i t A) = cos(tA) - i sin(tA) (Sec. 1, the Schroedinger case)
    from the oracle's cos/sin of tA; returns (U, info)."""
    A = _f64(A)
    C, S, info = cossin(float(t) * A, prec, m=m, s=s)
    return C - 1j * S, info


def unitary_gradient(A, t: float, G, m: int, s: int, prec: str = "double") -> np.ndarray:
    """d/dA of Re sum(conj(G) * U(A)) at fixed (2m, s) of tA.

    Re sum(conj(G) U) = <Re G, cos(tA)> + <-Im G, sin(tA)>, so by the chain
    rule the gradient is t times the cos/sin gradient at tA with the
    cotangents (Re G, -Im G)."""
    A = _f64(A)
    G = np.asarray(G, dtype=np.complex128)
    return float(t) * gradient(float(t) * A, G.real.copy(), -G.imag.copy(), m, s, prec)


def matmul(X, Y) -> np.ndarray:
    X = _f64(X)
    Y = _f64(Y)
    Z = np.zeros_like(X)
    _load().oracle_matmul(_ptr(X), _ptr(Y), _ptr(Z), X.shape[0])
    return Z


def frechet(A, E, m: int, s: int, prec: str = "double"):
    """Frechet derivatives L_cos(A, E), L_sin(A, E) of the approximant at fixed (2m, s).

    The approximant r is a polynomial in A, so r([[A, E], [0, A]]) carries
    L_r(A, E) in its upper-right block (Higham, Functions of Matrices, 2008,
    Thm. 3.6).  The block is exactly linear in E.
    """
    A = _f64(A)
    E = _f64(E)
    n = A.shape[0]
    X = np.zeros((2 * n, 2 * n))
    X[:n, :n] = A
    X[n:, n:] = A
    X[:n, n:] = E
    C, S, _ = cossin(X, prec, m=m, s=s)
    return C[:n, n:].copy(), S[:n, n:].copy()


def gradient(A, G_C, G_S, m: int, s: int, prec: str = "double") -> np.ndarray:
    """d/dA of <G_C, cos_r(A)> + <G_S, sin_r(A)> at fixed (2m, s).

    For a polynomial with real coefficients the adjoint of L_r(A, .) is
    L_r(A^T, .), so the gradient is L_cos(A^T, G_C) + L_sin(A^T, G_S).
    """
    A = _f64(A)
    Lc, _ = frechet(A.T, G_C, m, s, prec)
    _, Ls = frechet(A.T, G_S, m, s, prec)
    return Lc + Ls
