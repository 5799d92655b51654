"""The allocation-free 1-norm entry point (cossin_norm1_noalloc).

Some callers cannot allocate device memory (graph capture, pool-only
frameworks, loops that must not synchronise); this entry point runs the 1-norm
kernels on a static device scratch array instead.  It is checked against the
allocating entry point (cossin_norm1) through the C ABI, on two calls in a row
with different sizes so that the second call would see stale scratch from the
first if any word that must start at zero were not cleared.  This file is
collected last so that a run stopping at the first failure has run every
other test before it.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2010_00465_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu


def _noalloc(A, prec):
    L = _lib.lib()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.cossin_norm1_noalloc(ctypes.c_void_p(A.data_ptr()), A.shape[0], prec,
                                ctypes.c_void_p(out.data_ptr()), st)
    _lib.check(rc)
    torch.cuda.synchronize()
    return float(out.item())


def _alloc(A, prec):
    L = _lib.lib()
    res = ctypes.c_double()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _lib.check(L.cossin_norm1(ctypes.c_void_p(A.data_ptr()), A.shape[0], prec, ctypes.byref(res), st))
    return float(res.value)


@pytest.mark.parametrize("prec,dtype", [(_lib.CS_FP64, torch.float64), (_lib.CS_FP32, torch.float32)])
def test_noalloc_matches_allocating_entry_point_twice(prec, dtype):
    for n, idx in ((4096, 90), (1000, 91)):
        A = torch.from_numpy(inputs.matrix(n, "normal", None, index=idx)).to("cuda", dtype)
        got = _noalloc(A, prec)
        want = _alloc(A, prec)
        assert got == pytest.approx(want, rel=1e-14, abs=0.0), (n, got, want)


def test_noalloc_limits():
    L = _lib.lib()
    A = torch.zeros(4097, 4097, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.cossin_norm1_noalloc(ctypes.c_void_p(A.data_ptr()), 4097, _lib.CS_FP64,
                                ctypes.c_void_p(out.data_ptr()), st)
    assert rc == _lib.CS_EINVAL
    assert b"4096" in L.cossin_last_error()
    rc = L.cossin_norm1_noalloc(ctypes.c_void_p(A.data_ptr()), 0, _lib.CS_FP64,
                                ctypes.c_void_p(out.data_ptr()), st)
    assert rc == _lib.CS_OK
    torch.cuda.synchronize()
    assert float(out.item()) == 0.0
