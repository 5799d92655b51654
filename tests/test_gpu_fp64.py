"""Parity of the FP64 CUDA path with the FP64 oracle (relative Frobenius <= 1e-11).

Small and ragged sizes are compared element by element with the oracle at the
same (2m, s).  At n = 4096 (the benchmark's size and launch configuration) the
oracle is too slow for a dense matrix, so the comparison uses a permuted
block-diagonal matrix, whose cos and sin the oracle computes block by block,
and properties that hold at any size for a dense one.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2010_00465_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu
TOL64 = 1e-11


def relfro(X, Y):
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return float(np.linalg.norm(X - Y) / max(np.linalg.norm(Y), 1e-300))


def dev(A):
    return torch.from_numpy(np.ascontiguousarray(A)).cuda()


@pytest.mark.parametrize("n", [1, 2, 3, 7, 8, 64, 100, 127, 128, 129, 255, 300])
def test_norm1(n):
    A = inputs.matrix(n, "normal", None, index=40, sub=n)
    got = api.norm1(dev(A))
    assert got == pytest.approx(oracle.norm1(A), rel=1e-14)
    A32 = A.astype(np.float32)
    got32 = api.norm1(dev(A32), "fp32")
    assert got32 == pytest.approx(oracle.norm1(A32.astype(np.float64)), rel=1e-14)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_norm1_mixed_magnitudes(prec):
    """Columns whose entries span many binades, with zeros, negative zeros and
    subnormals (the column sums align every entry to the chunk's largest
    exponent in integer arithmetic, within 2^-48 of the exact sum)."""
    n = 300
    g = inputs.rng(44)
    lo, hi = (-60, 60) if prec == "fp64" else (-30, 30)
    A = g.standard_normal((n, n)) * np.exp2(g.integers(lo, hi, size=(n, n)))
    A[::7, ::3] = 0.0
    A[1::11, ::5] = -0.0
    tiny = np.finfo(np.float64 if prec == "fp64" else np.float32).tiny
    A[2::13, 1::4] = tiny * g.random((len(range(2, n, 13)), len(range(1, n, 4)))) * 0.5
    dt = np.float64 if prec == "fp64" else np.float32
    A = A.astype(dt)
    got = api.norm1(dev(A), prec)
    assert got == pytest.approx(oracle.norm1(A.astype(np.float64)), rel=1e-14)


def test_norm1_exact_and_extreme_values():
    g = inputs.rng(45)
    ints = g.integers(-2 ** 20, 2 ** 20, size=(257, 257)).astype(np.float64)
    assert api.norm1(dev(ints)) == float(np.abs(ints).sum(axis=0).max())  # integer sums are exact
    sub = np.full((70, 70), 5e-324) * g.integers(0, 1000, size=(70, 70))
    assert api.norm1(dev(sub)) == float(np.abs(sub).sum(axis=0).max())  # subnormals only: exact
    big = np.full((64, 64), 1e300)
    assert api.norm1(dev(big)) == pytest.approx(6.4e301, rel=1e-15)
    over = np.full((40, 40), 1e308)
    assert api.norm1(dev(over)) == np.inf  # the exact column sum overflows, as in FP64


def test_norm1_nan_inf():
    A = np.ones((50, 50))
    A[7, 9] = np.nan
    assert np.isnan(api.norm1(dev(A)))
    A[7, 9] = np.inf
    assert api.norm1(dev(A)) == np.inf


@pytest.mark.parametrize("n", [64, 1, 5, 127, 129, 200])
@pytest.mark.parametrize("nrm", [2.0 ** -6, 2.0 ** -4, 0.5, 1.0, 2.0, 8.0, 64.0])
def test_cossin_fp64_matches_oracle(n, nrm):
    A = inputs.matrix(n, "normal", nrm, index=41, sub=n)
    Co, So, info_o = oracle.cossin(A)
    C, S, info = api.cossin(dev(A), "fp64", m=info_o["m"], s=info_o["s"], return_info=True)
    assert (info["m"], info["s"]) == (info_o["m"], info_o["s"])
    assert relfro(C.cpu(), Co) <= TOL64
    assert relfro(S.cpu(), So) <= TOL64


@pytest.mark.parametrize("m", [4, 8, 9, 16, 24])
@pytest.mark.parametrize("s", [0, 1, 3])
def test_every_family_forced(m, s):
    A = inputs.matrix(96, "normal", 0.5 * 2 ** s, index=42, sub=m)
    Co, So, _ = oracle.cossin(A, m=m, s=s)
    C, S = api.cossin(dev(A), "fp64", m=m, s=s)
    assert relfro(C.cpu(), Co) <= TOL64
    assert relfro(S.cpu(), So) <= TOL64


@pytest.mark.parametrize("family", ["symmetric", "triangular", "uniform01", "uniform_pm", "nilpotent"])
@pytest.mark.parametrize("nrm", [2.0 ** -4, 1.0, 8.0, 64.0])
def test_families(family, nrm):
    A = inputs.matrix(130, family, nrm, index=43)
    Co, So, info_o = oracle.cossin(A)
    C, S, info = api.cossin(dev(A), "fp64", return_info=True)
    assert (info["m"], info["s"]) == (info_o["m"], info_o["s"])
    assert relfro(C.cpu(), Co) <= TOL64
    assert relfro(S.cpu(), So) <= TOL64


def test_auto_selection_matches_oracle():
    for nrm in (2.0 ** -4, 1.0, 8.0, 64.0, 3.3, 0.01):
        A = inputs.matrix(64, "normal", nrm, index=44)
        _, _, info = api.cossin(dev(A), "fp64", return_info=True)
        m, s = oracle.select(oracle.norm1(A), "double")
        assert (info["m"], info["s"]) == (m, s)
        assert info["products"] == {4: 3, 8: 4, 16: 6, 24: 7}[m] + 2 * s


def test_64x64_workload():
    """One 64 x 64 FP64 matrix, N(0,1) entries rescaled to ||A||_1 = 2."""
    A = inputs.matrix(64, "normal", 2.0, index=0)
    Co, So, info_o = oracle.cossin(A)
    C, S, info = api.cossin(dev(A), "fp64", return_info=True)
    assert (info["m"], info["s"]) == (24, 1) == (info_o["m"], info_o["s"])
    assert relfro(C.cpu(), Co) <= TOL64 and relfro(S.cpu(), So) <= TOL64


def test_jordan2_overscaling():
    for e in range(0, 9):
        A = inputs.jordan2(10.0 ** e) * (8.0 / (1 + 10.0 ** e))
        Co, So, info_o = oracle.cossin(A)
        C, S = api.cossin(dev(A), "fp64", m=info_o["m"], s=info_o["s"])
        assert np.abs(C.cpu().numpy() - Co).max() <= 1e-11 * max(1, np.abs(Co).max())
        assert np.abs(S.cpu().numpy() - So).max() <= 1e-11 * max(1, np.abs(So).max())


def test_edge_cases():
    z = torch.zeros(33, 33, dtype=torch.float64, device="cuda")
    C, S = api.cossin(z, "fp64")
    assert torch.equal(C, torch.eye(33, dtype=torch.float64, device="cuda"))
    assert torch.equal(S, torch.zeros_like(z))
    e = torch.zeros(0, 0, dtype=torch.float64, device="cuda")
    C, S = api.cossin(e, "fp64")
    assert C.shape == (0, 0)
    bad = torch.ones(8, 8, dtype=torch.float64, device="cuda")
    bad[1, 1] = float("nan")
    with pytest.raises(_lib.CossinError) as ex:
        api.cossin(bad, "fp64")
    assert ex.value.status == _lib.CS_ENONFINITE
    huge = torch.full((4, 4), 1e30, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.CossinError) as ex:
        api.cossin(huge, "fp64")
    assert ex.value.status == _lib.CS_ERANGE
    A = torch.randn(16, 16, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.CossinError) as ex:
        api.cossin(A, "fp64", out=(A, torch.empty_like(A)))
    assert ex.value.status == _lib.CS_EINVAL


def test_plain_entry_point_allocates_its_workspace():
    A = inputs.matrix(150, "normal", 8.0, index=45)
    Co, So, _ = oracle.cossin(A)
    Ad = dev(A)
    C = torch.empty_like(Ad)
    S = torch.empty_like(Ad)
    stream = torch.cuda.current_stream().cuda_stream
    import ctypes
    _lib.check(_lib.lib().cossin(ctypes.c_void_p(Ad.data_ptr()), 150, _lib.CS_FP64,
                                 ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(S.data_ptr()),
                                 ctypes.c_void_p(stream)))
    torch.cuda.synchronize()
    assert relfro(C.cpu(), Co) <= TOL64 and relfro(S.cpu(), So) <= TOL64


def test_host_tensors_round_trip():
    A = inputs.matrix(70, "normal", 3.0, index=46)
    Co, So, _ = oracle.cossin(A)
    C, S = api.cossin(torch.from_numpy(A), "fp64")
    assert not C.is_cuda
    assert relfro(C, Co) <= TOL64 and relfro(S, So) <= TOL64


# ------------------------------------------------------------ full size ---

def permuted_block_diagonal(n, block, nrm, index):
    """P diag(B_1..B_k) P^T with dense random blocks: cos and sin are
    P diag(f(B_i)) P^T exactly, and every block is small enough for the oracle."""
    g = inputs.rng(index, 0)
    k = n // block
    blocks = [inputs.matrix(block, "normal", None, index=index, sub=i + 1) for i in range(k)]
    worst = max(np.abs(B).sum(axis=0).max() for B in blocks)
    blocks = [B * (nrm / worst) for B in blocks]
    perm = g.permutation(n)
    A = np.zeros((n, n))
    for i, B in enumerate(blocks):
        idx = perm[i * block:(i + 1) * block]
        A[np.ix_(idx, idx)] = B
    return A, blocks, perm


@pytest.mark.parametrize("nrm", [2.0 ** -4, 1.0, 8.0, 64.0])
def test_full_size_block_diagonal(nrm):
    n, block = 4096, 64
    A, blocks, perm = permuted_block_diagonal(n, block, nrm, index=47)
    C, S, info = api.cossin(dev(A), "fp64", return_info=True)
    assert (info["m"], info["s"]) == oracle.select(oracle.norm1(A), "double")
    C = C.cpu().numpy()
    S = S.cpu().numpy()
    for i in list(range(0, len(blocks), 9)) + [len(blocks) - 1]:
        idx = perm[i * block:(i + 1) * block]
        Co, So, _ = oracle.cossin(blocks[i], m=info["m"], s=info["s"])
        assert relfro(C[np.ix_(idx, idx)], Co) <= TOL64
        assert relfro(S[np.ix_(idx, idx)], So) <= TOL64
    # everything outside the blocks is exactly zero
    mask = np.zeros((n, n), dtype=bool)
    for i in range(len(blocks)):
        idx = perm[i * block:(i + 1) * block]
        mask[np.ix_(idx, idx)] = True
    assert np.all(C[~mask] == 0.0) and np.all(S[~mask] == 0.0)


@pytest.mark.parametrize("family,nrm", [("normal", 8.0), ("normal", 64.0), ("triangular", 8.0)])
def test_full_size_dense_properties(family, nrm):
    """Dense n = 4096: cos^2 + sin^2 = I and commutation with A."""
    n = 4096
    A = dev(inputs.matrix(n, family, nrm, index=48))
    C, S = api.cossin(A, "fp64")
    I = torch.eye(n, dtype=torch.float64, device="cuda")
    R = C @ C + S @ S - I
    scale = (C @ C).norm() + (S @ S).norm()
    assert float(R.norm() / scale) <= TOL64
    K = C @ A - A @ C
    assert float(K.norm() / (C.norm() * A.norm())) <= TOL64


def test_full_size_symmetric_eigh():
    n = 4096
    A = dev(inputs.matrix(n, "symmetric", 8.0, index=49))
    w, V = torch.linalg.eigh(A)
    C, S = api.cossin(A, "fp64")
    Cr = (V * torch.cos(w)) @ V.T
    Sr = (V * torch.sin(w)) @ V.T
    assert float((C - Cr).norm() / Cr.norm()) <= TOL64
    assert float((S - Sr).norm() / Sr.norm()) <= TOL64


@pytest.mark.parametrize("pinned", [True, False])
def test_host_tensors_round_trip(pinned):
    """A CPU input is copied in, the results come back into the caller's CPU
    outputs (pinned: asynchronous copies on the call's stream, then a
    synchronisation), equal to the device call's results."""
    A = inputs.matrix(300, "normal", 8.0, index=46)
    C_dev, S_dev = api.cossin(dev(A), "fp64")
    host_A = torch.from_numpy(A)
    if pinned:
        host_A = host_A.pin_memory()
    out = (torch.empty(300, 300, dtype=torch.float64, pin_memory=pinned),
           torch.empty(300, 300, dtype=torch.float64, pin_memory=pinned))
    stream = torch.cuda.Stream()
    C, S = api.cossin(host_A, "fp64", out=out, stream=stream)
    assert C.data_ptr() == out[0].data_ptr() and S.data_ptr() == out[1].data_ptr()
    assert torch.equal(C, C_dev.cpu()) and torch.equal(S, S_dev.cpu())
    C2, S2 = api.cossin(torch.from_numpy(A), "fp64")
    assert torch.equal(C2, C) and torch.equal(S2, S)
    with pytest.raises(ValueError):
        api.cossin(host_A, "fp64", out=(torch.empty(3, 3, dtype=torch.float64), out[1]))


@pytest.mark.parametrize("n", [2304, 2500, 4096, 4100])
def test_product_with_split_last_wave(n):
    """The FP64 product whose last, partial wave of tiles runs as pieces split
    over K (2, 3 or 4 pieces at these orders on a 152-SM GB300, K a multiple
    of the piece length or not): sampled entries, most in the split tiles at
    the bottom of the matrix, against exactly summed dot products, within the
    K u bound of an FP64 product."""
    X = inputs.matrix(n, "normal", None, index=61, sub=n)
    Y = inputs.matrix(n, "normal", None, index=62, sub=n)
    P = api.matmul(dev(X), dev(Y), "fp64").cpu().numpy()
    g = inputs.rng(61, n)
    rows = np.concatenate([g.integers(0, n, 8), n - 1 - g.integers(0, min(n, 384), 24)])
    cols = g.integers(0, n, rows.size)
    for r, c in zip(rows, cols):
        terms = X[r, :] * Y[:, c]
        ref = math.fsum(terms.tolist())
        scale = math.fsum(np.abs(terms).tolist())
        assert abs(P[r, c] - ref) <= n * 2.0 ** -53 * scale, (r, c)
    assert api.fp64_product_launches(n, n, n) in (1, 2)


def test_product_launch_query():
    assert api.fp64_product_launches(64, 64, 64) == 1
    assert api.fp64_product_launches(0, 64, 64) == 0
    with pytest.raises(_lib.CossinError):
        api.fp64_product_launches(-1, 64, 64)
