"""Seeded synthetic inputs shaped like the test families of Sec. 4.

This module only draws numbers; it holds none of the method's arithmetic and
is shared by the tests, the benchmark, the CUDA path's callers and the oracle's
callers alike.  Every generator is NumPy PCG64 seeded with
``SEED_BASE + workload index (+ matrix index)`` and returns FP64 arrays whose
1-norm is rescaled to the requested value (the rescale is one multiplication,
so the norm lands within a few ulps of the target).

Families (Sec. 4 lists them for its 2500 test matrices):
  * ``normal``      iid N(0,1) entries ("randn")
  * ``uniform01``   iid U(0,1) entries ("rand")
  * ``uniform_pm``  iid U(-1/2, 1/2) entries
  * ``symmetric``   (X + X^T)/2 with X iid N(0,1)
  * ``triangular``  upper triangular, N(0,1) entries, strict upper part x10
                    (a strongly non-normal case)
  * ``nilpotent``   strictly upper triangular with a random number of nonzero
                    superdiagonals ("spdiags" + "rand")
  * ``jordan2``     the 2x2 matrix [[1, lam], [0, -1]] of Sec. 4
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 2010_00465

FAMILIES = ("normal", "uniform01", "uniform_pm", "symmetric", "triangular", "nilpotent")


def rng(index: int, sub: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([SEED_BASE + int(index), int(sub)]))


def _norm1(X: np.ndarray) -> float:
    return float(np.abs(X).sum(axis=0).max()) if X.size else 0.0


def rescale(X: np.ndarray, target_norm1: float | None) -> np.ndarray:
    if target_norm1 is None or X.size == 0:
        return X
    nrm = _norm1(X)
    if nrm == 0.0:
        return X
    return X * (float(target_norm1) / nrm)


def matrix(n: int, family: str = "normal", norm1: float | None = None, index: int = 0,
           sub: int = 0) -> np.ndarray:
    """One n x n FP64 matrix of ``family`` with ||A||_1 = ``norm1`` (if given)."""
    g = rng(index, sub)
    if family == "normal":
        X = g.standard_normal((n, n))
    elif family == "uniform01":
        X = g.random((n, n))
    elif family == "uniform_pm":
        X = g.random((n, n)) - 0.5
    elif family == "symmetric":
        Y = g.standard_normal((n, n))
        X = 0.5 * (Y + Y.T)
    elif family == "triangular":
        X = np.triu(g.standard_normal((n, n)))
        X = X + 9.0 * np.triu(X, 1)
    elif family == "nilpotent":
        X = np.zeros((n, n))
        if n > 1:
            bands = int(g.integers(1, n))
            for d in range(1, bands + 1):
                X += np.diag(g.random(n - d), d)
    else:
        raise ValueError("unknown family %r" % family)
    return np.ascontiguousarray(rescale(X, norm1))


def jordan2(lam: float) -> np.ndarray:
    """[[1, lam], [0, -1]] (Sec. 4, the overscaling family)."""
    return np.array([[1.0, float(lam)], [0.0, -1.0]])


def batch_shapes(count: int, n_lo: int = 8, n_hi: int = 256, norm_lo: float = 2.0 ** -6,
                 norm_hi: float = 2.0 ** 6, index: int = 3):
    """Sizes and norms for a batch: n and ||A||_1 log-uniform, half symmetric."""
    g = rng(index, 0)
    ns = np.rint(np.exp(g.uniform(np.log(n_lo), np.log(n_hi), size=count))).astype(np.int64)
    norms = np.exp(g.uniform(np.log(norm_lo), np.log(norm_hi), size=count))
    fams = np.where(np.arange(count) % 2 == 0, "symmetric", "normal")
    return ns, norms, fams


def batch(count: int, dtype=np.float32, index: int = 3, **kw):
    """A heterogeneous batch: list of arrays (n_i x n_i), plus the n and norms."""
    ns, norms, fams = batch_shapes(count, index=index, **kw)
    mats = [matrix(int(n), str(f), float(r), index=index, sub=i + 1).astype(dtype)
            for i, (n, r, f) in enumerate(zip(ns, norms, fams))]
    return mats, ns, norms


def hamiltonian_batch(count: int, n: int, terms: int = 4, index: int = 4):
    """A = H0 + sum_k u_k H_k, H_k = sym(N(0,1))/sqrt(n), u_k ~ U(-2, 2), and
    cotangents G_C, G_S ~ N(0,1): the control setting of the unitary
    propagator exp(-itA) = cos(tA) - i sin(tA) (Sec. 1, eq. unitary)."""
    g = rng(index, 0)
    H = []
    for _ in range(terms + 1):
        Y = g.standard_normal((n, n))
        H.append(0.5 * (Y + Y.T) / np.sqrt(n))
    u = g.uniform(-2.0, 2.0, size=(count, terms))
    A = np.empty((count, n, n))
    for b in range(count):
        A[b] = H[0] + np.tensordot(u[b], np.stack(H[1:]), axes=1)
    GC = g.standard_normal((count, n, n))
    GS = g.standard_normal((count, n, n))
    return A, GC, GS
