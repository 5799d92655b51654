"""Failure detection without a GPU fault: every wait in the tensor-core
kernels is bounded; an expired wait raises a device error word that the next
synchronising call reports as CS_ETIMEOUT, leaving the context usable.  The
self-test entry makes one such wait run out (an mbarrier nothing arrives at,
about 1 ms limit) through the same wait primitive and error word."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2010_00465_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu


def test_expired_wait_is_reported_once_and_the_context_stays_usable():
    A = inputs.matrix(48, "normal", 2.0, index=210)
    Ad = torch.from_numpy(A).cuda()
    api.cossin(Ad, "fp64")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert _lib.lib().cossin_selftest_wait_timeout(stream) == _lib.CS_OK
    with pytest.raises(_lib.CossinError) as ex:
        api.cossin(Ad, "fp64")
    assert ex.value.status == _lib.CS_ETIMEOUT
    assert b"bounded wait" in _lib.lib().cossin_last_error()
    # reported once: the word is cleared and the next calls run normally
    for prec, tol in (("fp64", 1e-11), ("fp32", 2e-5), ("fp64_emu", 1e-11)):
        x = Ad.float() if prec == "fp32" else Ad
        C, S = api.cossin(x, prec)
        Co, So, _ = oracle.cossin(x.double().cpu().numpy(), "single" if prec == "fp32" else "double")
        assert float(np.linalg.norm(C.double().cpu().numpy() - Co) / np.linalg.norm(Co)) <= tol
        assert float(np.linalg.norm(S.double().cpu().numpy() - So) / np.linalg.norm(So)) <= tol


def test_injected_allocation_failure_then_normal_calls():
    """A failed workspace allocation (injected on the host) returns CS_ENOMEM
    with no work queued; the next calls allocate and compute normally."""
    A = inputs.matrix(40, "normal", 3.0, index=211)
    Ad = torch.from_numpy(A).cuda()
    Co, So, _ = oracle.cossin(A)
    api.selftest_fail_next_alloc(1)
    with pytest.raises(_lib.CossinError) as ex:
        api.norm1(Ad)
    assert ex.value.status == _lib.CS_ENOMEM
    assert api.norm1(Ad) == pytest.approx(oracle.norm1(A), rel=1e-14)
    C = torch.empty_like(Ad)
    S = torch.empty_like(Ad)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    call = lambda: _lib.lib().cossin(ctypes.c_void_p(Ad.data_ptr()), 40, _lib.CS_FP64, ctypes.c_void_p(C.data_ptr()),
                                     ctypes.c_void_p(S.data_ptr()), stream)
    api.selftest_fail_next_alloc(1)
    assert call() == _lib.CS_ENOMEM
    assert call() == _lib.CS_OK
    api.device_status()
    assert float(np.linalg.norm(C.cpu().numpy() - Co) / np.linalg.norm(Co)) <= 1e-11
    assert float(np.linalg.norm(S.cpu().numpy() - So) / np.linalg.norm(So)) <= 1e-11
    G = torch.from_numpy(inputs.matrix(40, "normal", None, index=212)).cuda()
    api.selftest_fail_next_alloc(1)
    with pytest.raises(_lib.CossinError) as ex:
        api.cossin_backward(Ad, G, G)
    assert ex.value.status == _lib.CS_ENOMEM
    dA = api.cossin_backward(Ad, G, G)
    assert torch.isfinite(dA).all()
