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
