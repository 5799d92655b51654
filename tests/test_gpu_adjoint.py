"""The FP64 adjoint (reverse mode of the approximant at fixed (2m, s)).

Checked against (i) the oracle's gradient, read from the upper-right block of
the oracle's cos/sin of [[A^T, G], [0, A^T]] at the same (2m, s), and (ii)
central finite differences of the GPU forward pass at that (2m, s)."""
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
    return float(np.linalg.norm(X - Y) / np.linalg.norm(Y))


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("n", [1, 5, 17, 64, 130])
@pytest.mark.parametrize("family,nrm", [("normal", 0.05), ("normal", 1.0), ("normal", 8.0), ("triangular", 3.0),
                                        ("symmetric", 20.0)])
def test_matches_oracle_gradient(n, family, nrm):
    A = inputs.matrix(n, family, nrm, index=100, sub=n)
    GC = inputs.matrix(n, "normal", None, index=101, sub=n)
    GS = inputs.matrix(n, "normal", None, index=102, sub=n)
    dA, infos = api.cossin_backward(cuda(A), cuda(GC), cuda(GS), return_info=True)
    m, s = infos[0]["m"], infos[0]["s"]
    assert (m, s) == oracle.select(oracle.norm1(A), "double")
    ref = oracle.gradient(A, GC, GS, m, s)
    assert relfro(dA.cpu().numpy(), ref) <= TOL64


@pytest.mark.parametrize("m,s", [(4, 0), (8, 1), (16, 2), (24, 0), (24, 3), (9, 0), (9, 2)])
def test_every_family_forced(m, s):
    n = 40
    A = inputs.matrix(n, "normal", 0.5 * 2 ** s, index=103, sub=m)
    GC = inputs.matrix(n, "normal", None, index=104)
    GS = inputs.matrix(n, "normal", None, index=105)
    dA = api.cossin_backward(cuda(A), cuda(GC), cuda(GS), m=m, s=s)
    ref = oracle.gradient(A, GC, GS, m, s)
    assert relfro(dA.cpu().numpy(), ref) <= TOL64


def test_central_differences():
    n = 50
    A = inputs.matrix(n, "normal", 6.0, index=106)
    GC = inputs.matrix(n, "normal", None, index=107)
    GS = inputs.matrix(n, "normal", None, index=108)
    m, s = oracle.select(oracle.norm1(A), "double")
    dA = api.cossin_backward(cuda(A), cuda(GC), cuda(GS)).cpu().numpy()
    g = inputs.rng(109)
    for _ in range(3):
        E = g.standard_normal((n, n))
        h = 1e-6 * np.linalg.norm(A)
        Cp, Sp = api.cossin(cuda(A + h * E), "fp64", m=m, s=s)
        Cm, Sm = api.cossin(cuda(A - h * E), "fp64", m=m, s=s)
        fd = (np.sum(GC * (Cp - Cm).cpu().numpy()) + np.sum(GS * (Sp - Sm).cpu().numpy())) / (2 * h)
        an = float(np.sum(dA * E))
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1.0)


def test_forward_outputs_match_plain_path():
    A = inputs.matrix(70, "symmetric", 9.0, index=110)
    G = inputs.matrix(70, "normal", None, index=111)
    dA, C, S = api.cossin_backward(cuda(A), cuda(G), cuda(G), want_forward=True)
    C0, S0 = api.cossin(cuda(A), "fp64")
    assert relfro(C.cpu(), C0.cpu()) <= 1e-13 and relfro(S.cpu(), S0.cpu()) <= 1e-13


def test_autograd_function():
    A = cuda(inputs.matrix(24, "normal", 2.5, index=112)).requires_grad_(True)
    GC = cuda(inputs.matrix(24, "normal", None, index=113))
    GS = cuda(inputs.matrix(24, "normal", None, index=114))
    C, S = api.cossin_autograd(A)
    loss = (C * GC).sum() + (S * GS).sum()
    (g,) = torch.autograd.grad(loss, A)
    ref = api.cossin_backward(A.detach(), GC, GS)
    assert torch.allclose(g, ref, rtol=0, atol=0)
    # only one cotangent
    C, S = api.cossin_autograd(A)
    (g2,) = torch.autograd.grad((C * GC).sum(), A)
    ref2 = api.cossin_backward(A.detach(), GC, torch.zeros_like(GC))
    assert torch.equal(g2, ref2)


def test_autograd_gradcheck():
    A = cuda(inputs.matrix(4, "normal", 1.5, index=115)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda X: api.cossin_autograd(X), (A,), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_argument_errors():
    A = torch.zeros(3, 3, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.CossinError):
        api.cossin_backward(A, A, A, m=12, s=0)
    with pytest.raises(TypeError):
        api.cossin_backward(A.float(), A.float(), A.float())
    bad = A.clone()
    bad[0, 0] = float("nan")
    with pytest.raises(_lib.CossinError) as ex:
        api.cossin_backward(bad, A, A)
    assert ex.value.status == _lib.CS_ENONFINITE


def test_control_workload_sampled():
    """512 FP64 matrices n = 128, A = H0 + sum_k u_k H_k (random symmetric H_k,
    u_k ~ U(-2, 2)), random cotangents: one batched backward call; a sample is
    checked against the oracle's block-Frechet gradient, one against central
    differences, and the forward outputs against the plain FP64 path."""
    A, GC, GS = inputs.hamiltonian_batch(512, 128)
    dA, C, S = api.cossin_backward(cuda(A), cuda(GC), cuda(GS), want_forward=True)
    dA = dA.cpu().numpy()
    _, infos = api.cossin_backward(cuda(A[:8]), cuda(GC[:8]), cuda(GS[:8]), return_info=True)
    pairs = set()
    for b in range(512):
        pairs.add(oracle.select(oracle.norm1(A[b]), "double"))
    assert pairs <= {(24, 3), (16, 4), (24, 4), (24, 2), (16, 3)}
    for b in (0, 137, 511):
        m, s = oracle.select(oracle.norm1(A[b]), "double")
        ref = oracle.gradient(A[b], GC[b], GS[b], m, s)
        assert relfro(dA[b], ref) <= TOL64, b
    C0, S0 = api.cossin(cuda(A[5]), "fp64")
    assert relfro(C[5].cpu(), C0.cpu()) <= 1e-13
    b = 300
    m, s = oracle.select(oracle.norm1(A[b]), "double")
    E = inputs.rng(116).standard_normal((128, 128))
    h = 1e-6 * np.linalg.norm(A[b])
    Cp, Sp = api.cossin(cuda(A[b] + h * E), "fp64", m=m, s=s)
    Cm, Sm = api.cossin(cuda(A[b] - h * E), "fp64", m=m, s=s)
    fd = (np.sum(GC[b] * (Cp - Cm).cpu().numpy()) + np.sum(GS[b] * (Sp - Sm).cpu().numpy())) / (2 * h)
    assert abs(fd - float(np.sum(dA[b] * E))) <= 1e-7 * abs(fd)


@pytest.mark.parametrize("n", [1, 17, 64, 130])
@pytest.mark.parametrize("family,nrm", [("normal", 1.0), ("symmetric", 20.0), ("triangular", 3.0)])
def test_emulated_products_match_oracle_gradient(n, family, nrm):
    """The adjoint with its FP64 products emulated on the BF16 tensor cores
    (batched, transposed operands materialised) against the oracle's
    block-Frechet gradient."""
    A = inputs.matrix(n, family, nrm, index=120, sub=n)
    GC = inputs.matrix(n, "normal", None, index=121, sub=n)
    GS = inputs.matrix(n, "normal", None, index=122, sub=n)
    (dA, C, S), infos = api.cossin_backward(cuda(A), cuda(GC), cuda(GS), want_forward=True, return_info=True,
                                            prec="fp64_emu")
    m, s = infos[0]["m"], infos[0]["s"]
    ref = oracle.gradient(A, GC, GS, m, s)
    assert relfro(dA.cpu().numpy(), ref) <= TOL64
    Co, So, _ = oracle.cossin(A, m=m, s=s)
    assert relfro(C.cpu().numpy(), Co) <= TOL64 and relfro(S.cpu().numpy(), So) <= TOL64


def test_emulated_control_workload_sampled():
    A, GC, GS = inputs.hamiltonian_batch(512, 128)
    dA = api.cossin_backward(cuda(A), cuda(GC), cuda(GS), prec="fp64_emu").cpu().numpy()
    dA64 = api.cossin_backward(cuda(A), cuda(GC), cuda(GS)).cpu().numpy()
    assert relfro(dA, dA64) <= 1e-12
    for b in (3, 400):
        m, s = oracle.select(oracle.norm1(A[b]), "double")
        assert relfro(dA[b], oracle.gradient(A[b], GC[b], GS[b], m, s)) <= TOL64


def test_emulated_batched_split_last_round():
    """Four matrices of order 640 (200 emulated product tiles over a 152-SM
    grid, K over two 512-k chunks): the batched products' last round runs as
    K halves, spread over matrices of the batch; the gradient must match the
    native FP64 adjoint and, for one matrix, the oracle."""
    count, n = 4, 640
    A = np.stack([inputs.matrix(n, "normal", 3.0, index=125, sub=i + 1) for i in range(count)])
    GC = np.stack([inputs.matrix(n, "normal", None, index=126, sub=i + 1) for i in range(count)])
    GS = np.stack([inputs.matrix(n, "normal", None, index=127, sub=i + 1) for i in range(count)])
    dA = api.cossin_backward(cuda(A), cuda(GC), cuda(GS), prec="fp64_emu").cpu().numpy()
    dA64 = api.cossin_backward(cuda(A), cuda(GC), cuda(GS)).cpu().numpy()
    for b in range(count):
        assert relfro(dA[b], dA64[b]) <= 1e-11
    m, s = oracle.select(oracle.norm1(A[3]), "double")
    assert relfro(dA[3], oracle.gradient(A[3], GC[3], GS[3], m, s)) <= TOL64


def test_emulated_adjoint_argument_errors():
    A = torch.zeros(3, 3, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.CossinError) as ex:
        api.cossin_backward(A, A, A, prec="fp32")
    assert ex.value.status == _lib.CS_EINVAL


@pytest.mark.parametrize("prec", ["fp64", "fp64_emu"])
def test_caller_workspace_form_matches(prec):
    """cossin_backward_ws takes every buffer from the caller's workspace and
    gives the same gradient and forward outputs as the allocating form;
    a workspace below what the selected pairs need is refused before any work."""
    A, GC, GS = inputs.hamiltonian_batch(24, 48, index=9)
    Ad, GCd, GSd = cuda(A), cuda(GC), cuda(GS)
    (dA0, C0, S0), infos = api.cossin_backward(Ad, GCd, GSd, want_forward=True, return_info=True, prec=prec)
    max_s = max(i["s"] for i in infos)
    need = api.backward_workspace_size(24, 48, max_s, prec)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    dA1, C1, S1 = api.cossin_backward(Ad, GCd, GSd, want_forward=True, prec=prec, workspace=ws)
    assert torch.equal(dA0, dA1) and torch.equal(C0, C1) and torch.equal(S0, S1)
    ref = oracle.gradient(A[3], GC[3], GS[3], infos[3]["m"], infos[3]["s"])
    assert np.linalg.norm(dA1[3].cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-11
    small = torch.empty(need // 4, dtype=torch.uint8, device="cuda")
    with pytest.raises(_lib.CossinError) as ex:
        api.cossin_backward(Ad, GCd, GSd, prec=prec, workspace=small)
    assert ex.value.status == _lib.CS_EINVAL
