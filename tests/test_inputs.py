"""The seeded input generators (no method arithmetic): deterministic per
seed, norms on target, and each family's structure as stated in the input
recipe (the paper's Sec. 4 test families)."""
import numpy as np
import pytest

from paper_2010_00465_gb300 import inputs


def norm1(X):
    return float(np.abs(X).sum(axis=0).max())


@pytest.mark.parametrize("family", inputs.FAMILIES)
def test_deterministic_and_on_target_norm(family):
    A = inputs.matrix(50, family, 3.5, index=7, sub=2)
    B = inputs.matrix(50, family, 3.5, index=7, sub=2)
    assert np.array_equal(A, B)
    assert not np.array_equal(A, inputs.matrix(50, family, 3.5, index=7, sub=3))
    assert norm1(A) == pytest.approx(3.5, rel=8 * 2.0 ** -52)
    assert A.dtype == np.float64 and A.flags.c_contiguous


def test_family_structure():
    n = 40
    S = inputs.matrix(n, "symmetric", 2.0, index=8)
    assert np.array_equal(S, S.T)
    T = inputs.matrix(n, "triangular", None, index=8)
    assert not np.tril(T, -1).any() and np.tril(T).any()
    N = inputs.matrix(n, "nilpotent", 1.0, index=8)
    assert not np.tril(N).any()  # strictly upper triangular
    assert not np.linalg.matrix_power(N, n).any()  # nilpotent
    U = inputs.matrix(n, "uniform01", None, index=8)
    assert U.min() >= 0.0 and U.max() < 1.0
    P = inputs.matrix(n, "uniform_pm", None, index=8)
    assert P.min() >= -0.5 and P.max() < 0.5
    assert np.array_equal(inputs.jordan2(3.0), np.array([[1.0, 3.0], [0.0, -1.0]]))
    with pytest.raises(ValueError):
        inputs.matrix(4, "gallery")


def test_zero_and_empty():
    assert inputs.matrix(0, "normal", 1.0).shape == (0, 0)
    assert not inputs.rescale(np.zeros((3, 3)), 2.0).any()


def test_batched_workload_shapes():
    ns, norms, fams = inputs.batch_shapes(2000, index=3)
    assert ns.min() >= 8 and ns.max() <= 256
    assert norms.min() >= 2.0 ** -6 and norms.max() <= 2.0 ** 6
    assert (fams == "symmetric").sum() == 1000
    # log-uniform orders: about 60 % of the matrices have n <= 64 (ln 8 .. ln 64 of ln 8 .. ln 256)
    assert 0.55 < float((ns <= 64).mean()) < 0.65
    mats, ns2, _ = inputs.batch(6, index=3)
    assert [m.shape[0] for m in mats] == list(inputs.batch_shapes(6, index=3)[0])
    assert all(m.dtype == np.float32 for m in mats)


def test_control_hamiltonians():
    A, GC, GS = inputs.hamiltonian_batch(5, 12, index=4)
    assert A.shape == (5, 12, 12) and GC.shape == GS.shape == A.shape
    assert all(np.array_equal(a, a.T) for a in A)
    A2, _, _ = inputs.hamiltonian_batch(5, 12, index=4)
    assert np.array_equal(A, A2)
