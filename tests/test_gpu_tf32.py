"""Parity of the tensor-core paths with the FP64 oracle.

CS_FP32: FP32 in/out, single table, FP64 intermediates, every product a
four-slice BF16 tcgen05 product; CS_SPLIT_TF32: FP64 in/out, single table,
Taylor chain on the four-pass TF32 tensor-core kernel with FP64 intermediates,
double-angle steps in FP64 (CS_SPLIT_EMU: those emulated on the BF16 tensor
cores); CS_SPLIT_BF16: the Taylor chain as four-slice BF16 products, the
double-angle steps as eight-slice ones.  All are compared with the oracle run
on the same input (FP32 inputs upcast exactly) at the same (2m, s) with the
single table; the bound is 2e-5 relative Frobenius for ||A||_1 <= 64 at every
order, 1 x 1 included.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2010_00465_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu
TOL32 = 2e-5


def relfro(X, Y):
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return float(np.linalg.norm(X - Y) / max(np.linalg.norm(Y), 1e-300))


def run(A, prec, **kw):
    dt = torch.float32 if prec == "fp32" else torch.float64
    Ad = torch.from_numpy(np.ascontiguousarray(A)).to("cuda", dt)
    C, S, info = api.cossin(Ad, prec, return_info=True, **kw)
    return C.double().cpu().numpy(), S.double().cpu().numpy(), info


@pytest.mark.parametrize("prec", ["fp32", "split_tf32", "split_emu", "split_bf16"])
@pytest.mark.parametrize("n", [1, 5, 33, 64, 100, 128, 129, 192, 255, 256, 257, 300])
@pytest.mark.parametrize("nrm", [2.0 ** -6, 2.0 ** -4, 1.0, 8.0, 30.0, 64.0])
@pytest.mark.parametrize("family", ["normal", "symmetric"])
def test_matches_oracle(prec, n, nrm, family):
    A = inputs.matrix(n, family, nrm, index=60, sub=n)
    if prec == "fp32":
        A = A.astype(np.float32).astype(np.float64)
    Co, So, info_o = oracle.cossin(A, "single")
    C, S, info = run(A, prec, m=info_o["m"], s=info_o["s"])
    assert info["table"] == 1
    assert relfro(C, Co) <= TOL32, relfro(C, Co)
    assert relfro(S, So) <= TOL32, relfro(S, So)


@pytest.mark.parametrize("prec", ["fp32", "split_tf32", "split_emu", "split_bf16"])
@pytest.mark.parametrize("m", [4, 8, 9, 16, 24])
@pytest.mark.parametrize("s", [0, 2])
def test_every_family_forced(prec, m, s):
    A = inputs.matrix(160, "normal", 2.0 * 2 ** s, index=61, sub=m)
    if prec == "fp32":
        A = A.astype(np.float32).astype(np.float64)
    Co, So, _ = oracle.cossin(A, "single", m=m, s=s)
    C, S, _ = run(A, prec, m=m, s=s)
    assert relfro(C, Co) <= TOL32 and relfro(S, So) <= TOL32


@pytest.mark.parametrize("prec", ["fp32", "split_tf32", "split_emu", "split_bf16"])
@pytest.mark.parametrize("family", ["symmetric", "triangular", "uniform01", "uniform_pm", "nilpotent"])
def test_families(prec, family):
    for nrm in (2.0 ** -4, 1.0, 8.0, 64.0):
        A = inputs.matrix(192, family, nrm, index=62)
        if prec == "fp32":
            A = A.astype(np.float32).astype(np.float64)
        Co, So, info_o = oracle.cossin(A, "single")
        C, S, info = run(A, prec)
        assert (info["m"], info["s"]) == (info_o["m"], info_o["s"])
        assert relfro(C, Co) <= TOL32 and relfro(S, So) <= TOL32, (family, nrm)


@pytest.mark.parametrize("prec", ["fp32", "split_tf32", "split_emu", "split_bf16"])
def test_accuracy_against_double_oracle(prec):
    """Against the true function (oracle, double table) the error stays FP32-level."""
    for nrm in (0.1, 1.0, 8.0, 64.0):
        A = inputs.matrix(128, "normal", nrm, index=63)
        if prec == "fp32":
            A = A.astype(np.float32).astype(np.float64)
        Co, So, _ = oracle.cossin(A, "double")
        C, S, _ = run(A, prec)
        assert relfro(C, Co) <= TOL32 and relfro(S, So) <= TOL32


def test_fp32_edge_cases():
    z = torch.zeros(40, 40, dtype=torch.float32, device="cuda")
    C, S = api.cossin(z, "fp32")
    assert torch.equal(C, torch.eye(40, device="cuda")) and torch.equal(S, torch.zeros_like(z))
    e = torch.zeros(0, 0, dtype=torch.float32, device="cuda")
    C, S = api.cossin(e, "fp32")
    assert C.shape == (0, 0)
    bad = torch.ones(8, 8, device="cuda")
    bad[0, 3] = float("inf")
    with pytest.raises(_lib.CossinError) as ex:
        api.cossin(bad, "fp32")
    assert ex.value.status == _lib.CS_ENONFINITE
    with pytest.raises(TypeError):
        api.cossin(torch.ones(4, 4, dtype=torch.float64, device="cuda"), "fp32")


def test_device_status_clean():
    import ctypes
    assert _lib.lib().cossin_device_status(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0


# ------------------------------------------------------------ full size ---

def _block_case(n, block, nrm, index):
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


@pytest.mark.parametrize("prec", ["fp32", "split_tf32", "split_emu", "split_bf16"])
@pytest.mark.parametrize("nrm", [2.0 ** -4, 1.0, 8.0, 64.0])
def test_full_size_block_diagonal(prec, nrm):
    n, block = 4096, 64
    A, blocks, perm = _block_case(n, block, nrm, index=64)
    if prec == "fp32":
        A = A.astype(np.float32).astype(np.float64)
    C, S, info = run(A, prec)
    assert (info["m"], info["s"]) == oracle.select(oracle.norm1(A), "single")
    for i in list(range(0, len(blocks), 9)) + [len(blocks) - 1]:
        idx = perm[i * block:(i + 1) * block]
        Co, So, _ = oracle.cossin(A[np.ix_(idx, idx)], "single", m=info["m"], s=info["s"])
        assert relfro(C[np.ix_(idx, idx)], Co) <= TOL32
        assert relfro(S[np.ix_(idx, idx)], So) <= TOL32


_FULL_CASES = [("normal", 2.0 ** -4), ("normal", 1.0), ("normal", 8.0), ("normal", 64.0), ("symmetric", 8.0),
               ("triangular", 8.0)]
@pytest.mark.parametrize("prec", ["fp32", "split_tf32", "split_emu", "split_bf16"])
@pytest.mark.parametrize("family,nrm", _FULL_CASES)
def test_full_size_against_fp64_path(prec, family, nrm):
    """n = 4096 dense: the FP32 and split paths against the FP64 path, which
    the FP64 tests pin to the oracle within 1e-11 at this size; 2e-5 is the
    FP32 target for ||A||_1 <= 64."""
    n = 4096
    A = inputs.matrix(n, family, nrm, index=66)
    A32 = A.astype(np.float32).astype(np.float64)
    C64, S64 = api.cossin(torch.from_numpy(A32).cuda(), "fp64")
    dt = torch.float32 if prec == "fp32" else torch.float64
    C, S = api.cossin(torch.from_numpy(A32).to("cuda", dt), prec)
    ec = float((C.double() - C64).norm() / C64.norm())
    es = float((S.double() - S64).norm() / S64.norm())
    assert ec <= TOL32 and es <= TOL32, (prec, family, nrm, ec, es)


@pytest.mark.parametrize("prec", ["fp32", "split_tf32", "split_emu", "split_bf16"])
@pytest.mark.parametrize("family,nrm", [("normal", 8.0), ("normal", 64.0), ("triangular", 8.0), ("symmetric", 8.0)])
def test_full_size_dense_properties(prec, family, nrm):
    n = 4096
    A = inputs.matrix(n, family, nrm, index=65)
    dt = torch.float32 if prec == "fp32" else torch.float64
    Ad = torch.from_numpy(A).to("cuda", dt)
    C, S = api.cossin(Ad, prec)
    Cd, Sd, Ad = C.double(), S.double(), Ad.double()
    I = torch.eye(n, dtype=torch.float64, device="cuda")
    R = Cd @ Cd + Sd @ Sd - I
    assert float(R.norm() / ((Cd @ Cd).norm() + (Sd @ Sd).norm())) <= TOL32
    K = Cd @ Ad - Ad @ Cd
    assert float(K.norm() / (Cd.norm() * Ad.norm())) <= TOL32
    if family == "symmetric":
        w, V = torch.linalg.eigh(Ad)
        Cr = (V * torch.cos(w)) @ V.T
        assert float((Cd - Cr).norm() / Cr.norm()) <= TOL32


@pytest.mark.parametrize("prec", ["split_tf32", "split_emu", "split_bf16"])
@pytest.mark.parametrize("nrm", [1.0, 64.0])
def test_split_n8192_block_diagonal(prec, nrm):
    """The split workload's larger order, n = 8192: a permuted block-diagonal
    matrix, sampled 64-blocks against the oracle at the same (2m, s)."""
    n, block = 8192, 64
    A, blocks, perm = _block_case(n, block, nrm, index=67)
    C, S, info = run(A, prec)
    assert (info["m"], info["s"]) == oracle.select(oracle.norm1(A), "single")
    for i in list(range(0, len(blocks), 23)) + [len(blocks) - 1]:
        idx = perm[i * block:(i + 1) * block]
        Co, So, _ = oracle.cossin(A[np.ix_(idx, idx)], "single", m=info["m"], s=info["s"])
        assert relfro(C[np.ix_(idx, idx)], Co) <= TOL32
        assert relfro(S[np.ix_(idx, idx)], So) <= TOL32
