"""Parity of the c(t^2 A), s(t, A) path (Sec. 2.2) with the oracle.

Small and ragged orders are compared element by element with the oracle at
the same (family, sigma) -- relative Frobenius 1e-11 for FP64, the FP32 bound
of the cos/sin tests (at ||A||_1 read as sqrt(||t^2 A||_1), the size of the
cosine's argument) for the two single-table forms.  At n = 4096 the oracle
runs on the blocks of a permuted block-diagonal matrix, and a dense matrix
A = X^2 is checked against the cos/sin path: c(t^2 X^2) = cos(tX) and
X s(t, X^2) = sin(tX).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2010_00465_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu
TOL64 = 1e-11
TOL32 = 2e-5


def relfro(X, Y):
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return float(np.linalg.norm(X - Y) / max(np.linalg.norm(Y), 1e-300))


def dev(A, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(A)).to(dtype).cuda()


def step_for(A, normB, sign=1.0):
    """t with ||t^2 A||_1 = normB."""
    return sign * math.sqrt(normB / oracle.norm1(A))


def laplacian(n):
    """1-D Dirichlet Laplacian (n + 1)^2 tridiag(-1, 2, -1): the matrix of the
    semi-discrete wave equation u'' + A u = 0 that motivates Sec. 2.2."""
    A = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    return A * (n + 1) ** 2


@pytest.mark.parametrize("n", [1, 5, 64, 129, 200])
@pytest.mark.parametrize("normB", [1e-3, 0.05, 1.0, 10.0, 100.0, 1000.0])
@pytest.mark.parametrize("family", ["normal", "symmetric"])
def test_fp64_matches_oracle(n, normB, family):
    A = inputs.matrix(n, family, 1.0, index=150, sub=n)
    t = step_for(A, normB, -1.0 if n == 129 else 1.0)
    Co, So, io = oracle.cs(A, t)
    C, S, info = api.cossin_cs(dev(A), t, "fp64", return_info=True)
    assert (info["m"], info["s"]) == (io["m"], io["s"]) == oracle.cs_select(io["norm1"], "double")
    assert info["norm1"] == pytest.approx(io["norm1"], rel=1e-14)
    assert info["products"] == io["products"]
    assert relfro(C.cpu(), Co) <= TOL64
    assert relfro(S.cpu(), So) <= TOL64


@pytest.mark.parametrize("fam", [0, 1, 2, 3])
@pytest.mark.parametrize("sigma", [0, 1, 3])
def test_every_family_forced(fam, sigma):
    n = 40
    A = inputs.matrix(n, "normal", 1.0, index=151, sub=4 * fam + sigma)
    t = step_for(A, 0.5 * 4.0 ** sigma)
    Co, So, io = oracle.cs(A, t, family=fam, sigma=sigma)
    C, S, info = api.cossin_cs(dev(A), t, "fp64", family=fam, sigma=sigma, return_info=True)
    assert (info["m"], info["s"], info["products"]) == (fam, sigma, io["products"])
    assert relfro(C.cpu(), Co) <= TOL64
    assert relfro(S.cpu(), So) <= TOL64


@pytest.mark.parametrize("prec", ["fp32", "split_tf32", "split_emu", "split_bf16"])
@pytest.mark.parametrize("n", [1, 3, 5, 33, 64, 129, 200])
@pytest.mark.parametrize("normB", [0.01, 1.0, 20.0, 300.0, 900.0, 4096.0])
def test_single_table_forms_match_oracle(prec, n, normB):
    A = inputs.matrix(n, "normal", 1.0, index=152, sub=n).astype(np.float32).astype(np.float64)
    t = step_for(A, normB)
    Co, So, io = oracle.cs(A, t, "single")
    dt = torch.float32 if prec == "fp32" else torch.float64
    C, S, info = api.cossin_cs(dev(A, dt), t, prec, return_info=True)
    assert (info["m"], info["s"]) == (io["m"], io["s"])
    assert info["table"] == 1
    assert relfro(C.double().cpu(), Co) <= TOL32
    assert relfro(S.double().cpu(), So) <= TOL32


@pytest.mark.parametrize("prec", ["fp32", "split_tf32", "split_emu", "split_bf16"])
@pytest.mark.parametrize("fam", [0, 1, 2, 3])
def test_single_table_every_family(prec, fam):
    n = 96
    A = inputs.matrix(n, "symmetric", 1.0, index=153, sub=fam).astype(np.float32).astype(np.float64)
    t = step_for(A, 2.0)
    sigma = 1
    Co, So, _ = oracle.cs(A, t, "single", family=fam, sigma=sigma)
    dt = torch.float32 if prec == "fp32" else torch.float64
    C, S = api.cossin_cs(dev(A, dt), t, prec, family=fam, sigma=sigma)
    assert relfro(C.double().cpu(), Co) <= TOL32
    assert relfro(S.double().cpu(), So) <= TOL32


def test_wave_equation_laplacian():
    """One step of u'' + A u = 0 with the 1-D Laplacian (n = 127): C u0 + S v0
    against the oracle, and against the eigen-decomposition's exact solution."""
    n = 127
    A = laplacian(n)
    t = 0.7 / (n + 1)
    Co, So, io = oracle.cs(A, t)
    C, S, info = api.cossin_cs(dev(A), t, "fp64", return_info=True)
    assert (info["m"], info["s"]) == (io["m"], io["s"])
    assert relfro(C.cpu(), Co) <= TOL64 and relfro(S.cpu(), So) <= TOL64
    lam, V = np.linalg.eigh(A)
    w = np.sqrt(lam)
    Ce = (V * np.cos(t * w)) @ V.T
    Se = (V * (np.sin(t * w) / w)) @ V.T
    assert relfro(C.cpu(), Ce) <= 1e-12 and relfro(S.cpu(), Se) <= 1e-12


def test_degenerate_cases():
    n = 33
    A = inputs.matrix(n, "normal", 3.0, index=154)
    eye = np.eye(n)
    for prec, dt in (("fp64", torch.float64), ("fp32", torch.float32), ("split_tf32", torch.float64)):
        # t = 0: c = I, s = 0 exactly
        C, S, info = api.cossin_cs(dev(A, dt), 0.0, prec, return_info=True)
        assert info["norm1"] == 0.0 and info["s"] == 0
        assert np.array_equal(C.double().cpu().numpy(), eye)
        assert not S.double().cpu().numpy().any()
        # A = 0: c = I, s = t I exactly
        C, S = api.cossin_cs(dev(np.zeros((n, n)), dt), 0.75, prec)
        assert np.array_equal(C.double().cpu().numpy(), eye)
        assert np.array_equal(S.double().cpu().numpy(), 0.75 * eye)
    # n = 0
    C, S, info = api.cossin_cs(torch.zeros(0, 0, dtype=torch.float64, device="cuda"), 1.0, "fp64",
                               return_info=True)
    assert C.shape == (0, 0) and info["products"] == 0


def test_argument_errors():
    A = dev(inputs.matrix(8, "normal", 1.0, index=155))
    for bad_t in (float("nan"), float("inf")):
        with pytest.raises(_lib.CossinError) as ex:
            api.cossin_cs(A, bad_t, "fp64")
        assert ex.value.status == _lib.CS_EINVAL
    with pytest.raises(_lib.CossinError) as ex:
        api.cossin_cs(A, 1.0, "fp64", family=4, sigma=0)
    assert ex.value.status == _lib.CS_EINVAL
    with pytest.raises(_lib.CossinError) as ex:
        api.cossin_cs(A, 1.0, "fp64", family=1)
    assert ex.value.status == _lib.CS_EINVAL
    N = A.clone()
    N[2, 3] = float("nan")
    with pytest.raises(_lib.CossinError) as ex:
        api.cossin_cs(N, 1.0, "fp64")
    assert ex.value.status == _lib.CS_ENONFINITE
    with pytest.raises(_lib.CossinError) as ex:
        api.cossin_cs(A, 1e200, "fp64")
    assert ex.value.status == _lib.CS_ENONFINITE
    with pytest.raises(_lib.CossinError) as ex:
        api.cossin_cs(A, 1e40, "fp64")
    assert ex.value.status == _lib.CS_ERANGE


def _block_case(n, block, normB, index):
    g = inputs.rng(index)
    perm = g.permutation(n)
    blocks = [inputs.matrix(block, "normal", 1.0, index=index, sub=i) for i in range(n // block)]
    A = np.zeros((n, n))
    for i, B in enumerate(blocks):
        idx = perm[i * block:(i + 1) * block]
        A[np.ix_(idx, idx)] = B
    return A, perm, math.sqrt(normB / oracle.norm1(A))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split_tf32"])
@pytest.mark.parametrize("normB", [0.1, 30.0])
def test_full_size_block_diagonal(prec, normB):
    n, block = 4096, 64
    A, perm, t = _block_case(n, block, normB, index=156)
    table = "double" if prec == "fp64" else "single"
    if prec == "fp32":
        A = A.astype(np.float32).astype(np.float64)
    dt = torch.float32 if prec == "fp32" else torch.float64
    C, S, info = api.cossin_cs(dev(A, dt), t, prec, return_info=True)
    assert (info["m"], info["s"]) == oracle.cs_select(t * t * oracle.norm1(A), table)
    C = C.double().cpu().numpy()
    S = S.double().cpu().numpy()
    tol = TOL64 if prec == "fp64" else TOL32
    for i in list(range(0, n // block, 11)) + [n // block - 1]:
        idx = perm[i * block:(i + 1) * block]
        Co, So, _ = oracle.cs(A[np.ix_(idx, idx)], t, table, family=info["m"], sigma=info["s"])
        assert relfro(C[np.ix_(idx, idx)], Co) <= tol
        assert relfro(S[np.ix_(idx, idx)], So) <= tol
    # off-block entries stay exactly zero
    mask = np.ones((n, n), dtype=bool)
    for i in range(n // block):
        idx = perm[i * block:(i + 1) * block]
        mask[np.ix_(idx, idx)] = False
    assert not C[mask].any() and not S[mask].any()


@pytest.mark.parametrize("normX", [0.5, 6.0])
def test_full_size_dense_squares(normX):
    """n = 4096 dense, A = X^2: c(t^2 A) = cos(tX) and X s(t, A) = sin(tX),
    with cos and sin from the FP64 cos/sin path (pinned to the oracle)."""
    n = 4096
    X = dev(inputs.matrix(n, "normal", normX, index=157))
    A = X @ X
    t = 1.0
    C, S = api.cossin_cs(A, t, "fp64")
    Cx, Sx = api.cossin(X, "fp64")
    assert relfro(C.cpu(), Cx.cpu()) <= 1e-10
    assert relfro((X @ S).cpu(), Sx.cpu()) <= 1e-10
