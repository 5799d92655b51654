"""The propagator exp(-i t A) = cos(tA) - i sin(tA) and its adjoint on the GPU,
against the oracle at the same (2m, s) of tA."""
import numpy as np
import pytest
import torch

import oracle
from paper_2010_00465_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu
TOL64 = 1e-11
TOL32 = 2e-5


def relfro(X, Y):
    X = np.asarray(X)
    Y = np.asarray(Y)
    return float(np.linalg.norm(X - Y) / max(np.linalg.norm(Y), 1e-300))


def dev(A, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(A)).to(dtype).cuda()


@pytest.mark.parametrize("n", [1, 7, 64, 129, 200])
@pytest.mark.parametrize("t", [0.01, 1.0, -3.0, 20.0])
@pytest.mark.parametrize("family", ["symmetric", "normal"])
def test_fp64_matches_oracle(n, t, family):
    A = inputs.matrix(n, family, 2.0, index=180, sub=n)
    Uo, io = oracle.unitary(A, t)
    U, info = api.unitary(dev(A), t, "fp64", return_info=True)
    assert U.dtype == torch.complex128
    assert (info["m"], info["s"]) == (io["m"], io["s"])
    assert info["norm1"] == pytest.approx(abs(t) * oracle.norm1(A), rel=1e-14)
    assert relfro(U.cpu().numpy(), Uo) <= TOL64


@pytest.mark.parametrize("prec", ["fp32", "split_tf32"])
@pytest.mark.parametrize("n", [5, 96, 257])
@pytest.mark.parametrize("t", [0.1, 4.0])
def test_single_table_forms(prec, n, t):
    A = inputs.matrix(n, "symmetric", 2.0, index=181, sub=n).astype(np.float32).astype(np.float64)
    Uo, io = oracle.unitary(A, t, "single")
    dt = torch.float32 if prec == "fp32" else torch.float64
    U, info = api.unitary(dev(A, dt), t, prec, return_info=True)
    assert U.dtype == (torch.complex64 if prec == "fp32" else torch.complex128)
    assert (info["m"], info["s"]) == (io["m"], io["s"])
    assert relfro(U.cpu().numpy().astype(np.complex128), Uo) <= TOL32


def test_unitarity_at_full_size():
    """n = 4096 symmetric: U U^H = I (sampled rows) and U(2t) = U(t)^2."""
    n = 4096
    A = dev(inputs.matrix(n, "symmetric", 8.0, index=182))
    U1 = api.unitary(A, 0.5, "fp64")
    U2 = api.unitary(A, 1.0, "fp64")
    rows = torch.tensor([0, 1, 777, 2048, 4095], device="cuda")
    P = U1[rows] @ U1.conj().T
    I = torch.zeros_like(P)
    I[torch.arange(5), rows] = 1.0
    assert float((P - I).abs().max()) <= 1e-12
    assert float((U1 @ U1 - U2).norm() / U2.norm()) <= 1e-12


@pytest.mark.parametrize("n", [3, 40, 130])
@pytest.mark.parametrize("t", [0.5, -2.5])
def test_backward_matches_oracle(n, t):
    A = inputs.matrix(n, "symmetric", 3.0, index=183, sub=n)
    g = inputs.rng(184)
    G = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    (dA, U), infos = api.unitary_backward(dev(A), t, torch.from_numpy(G).cuda(), want_forward=True,
                                          return_info=True)
    m, s = infos[0]["m"], infos[0]["s"]
    assert (m, s) == oracle.select(abs(t) * oracle.norm1(A), "double")
    ref = oracle.unitary_gradient(A, t, G, m, s)
    assert relfro(dA.cpu().numpy(), ref) <= TOL64
    Uo, _ = oracle.unitary(A, t)
    assert relfro(U.cpu().numpy(), Uo) <= TOL64


def test_backward_batched_control_workload():
    """The control setting A = H0 + sum u_k H_k (512 x n = 128), one call; a
    sample against the oracle and one against central differences of the
    GPU forward pass."""
    A, GC, GS = inputs.hamiltonian_batch(512, 128)
    G = GC + 1j * GS
    t = 0.8
    dA = api.unitary_backward(dev(A), t, torch.from_numpy(G).cuda()).cpu().numpy()
    for b in (0, 311):
        m, s = oracle.select(t * oracle.norm1(A[b]), "double")
        ref = oracle.unitary_gradient(A[b], t, G[b], m, s)
        assert relfro(dA[b], ref) <= TOL64, b
    b = 99
    m, s = oracle.select(t * oracle.norm1(A[b]), "double")
    E = inputs.rng(185).standard_normal((128, 128))
    h = 1e-6 * np.linalg.norm(A[b])
    Up = api.unitary(dev(A[b] + h * E), t, "fp64", m=m, s=s).cpu().numpy()
    Um = api.unitary(dev(A[b] - h * E), t, "fp64", m=m, s=s).cpu().numpy()
    fd = float(np.real(np.sum(np.conj(G[b]) * (Up - Um)))) / (2 * h)
    assert abs(fd - float(np.sum(dA[b] * E))) <= 1e-7 * abs(fd)


def test_autograd():
    A = dev(inputs.matrix(12, "symmetric", 1.5, index=186)).requires_grad_(True)
    g = inputs.rng(187)
    G = torch.from_numpy(g.standard_normal((12, 12)) + 1j * g.standard_normal((12, 12))).cuda()
    U = api.unitary_autograd(A, 0.9)
    loss = (torch.conj(G) * U).real.sum()
    (dA,) = torch.autograd.grad(loss, A)
    ref = api.unitary_backward(A.detach(), 0.9, G)
    assert torch.equal(dA, ref)
    B = dev(inputs.matrix(4, "normal", 1.0, index=188)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda X: api.unitary_autograd(X, 0.6), (B,), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_edges_and_errors():
    A = dev(inputs.matrix(6, "normal", 1.0, index=189))
    U = api.unitary(A, 0.0, "fp64")
    assert torch.equal(U, torch.eye(6, dtype=torch.complex128, device="cuda"))
    Z = api.unitary(torch.zeros(0, 0, dtype=torch.float64, device="cuda"), 1.0, "fp64")
    assert Z.shape == (0, 0)
    with pytest.raises(_lib.CossinError) as ex:
        api.unitary(A, float("nan"), "fp64")
    assert ex.value.status == _lib.CS_EINVAL
    with pytest.raises(_lib.CossinError) as ex:
        api.unitary(A, 1e300, "fp64")
    assert ex.value.status in (_lib.CS_ENONFINITE, _lib.CS_ERANGE)
    G = torch.zeros(6, 6, dtype=torch.complex128, device="cuda")
    with pytest.raises(_lib.CossinError):
        api.unitary_backward(A, float("inf"), G)
