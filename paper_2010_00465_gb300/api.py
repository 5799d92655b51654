"""PyTorch-facing calls of the library.

PyTorch supplies device memory and the current stream; every step of the
method runs in the library's CUDA kernels behind the C ABI.  There is no CPU
fallback: without the built library or a GPU these calls raise.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import CsInfo, check, lib

PRECISIONS = {"fp64": _lib.CS_FP64, "fp32": _lib.CS_FP32, "split_tf32": _lib.CS_SPLIT_TF32}
_DTYPE = {_lib.CS_FP64: torch.float64, _lib.CS_FP32: torch.float32, _lib.CS_SPLIT_TF32: torch.float64}


def _prec(prec, A=None) -> int:
    if prec is None:
        if A is None:
            raise ValueError("precision needed")
        prec = "fp32" if A.dtype == torch.float32 else "fp64"
    if isinstance(prec, str):
        return PRECISIONS[prec]
    return int(prec)


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _check_matrix(A: torch.Tensor, p: int) -> int:
    if A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be square, got %r" % (tuple(A.shape),))
    if A.dtype != _DTYPE[p]:
        raise TypeError("precision %d needs %s input, got %s" % (p, _DTYPE[p], A.dtype))
    if not A.is_cuda:
        raise ValueError("A must be a CUDA tensor")
    if not A.is_contiguous():
        raise ValueError("A must be contiguous (row-major)")
    return int(A.shape[0])


def workspace_size(n: int, prec="fp64") -> int:
    out = ctypes.c_size_t()
    check(lib().cossin_workspace_size(int(n), _prec(prec), ctypes.byref(out)))
    return int(out.value)


def norm1(A: torch.Tensor, prec=None, stream=None) -> float:
    """||A||_1 computed on the device (FP64 accumulation)."""
    p = _prec(prec, A)
    n = _check_matrix(A, p)
    out = ctypes.c_double()
    check(lib().cossin_norm1(ctypes.c_void_p(A.data_ptr()), n, p, ctypes.byref(out), _stream_ptr(stream)))
    return float(out.value)


def select(norm: float, table: int):
    """(2m, s) for ||A||_1 = norm; table 0 = double (Table 1), 1 = single (Table 2)."""
    m = ctypes.c_int32()
    s = ctypes.c_int32()
    check(lib().cossin_select(float(norm), int(table), ctypes.byref(m), ctypes.byref(s)))
    return m.value, s.value


def cossin(A: torch.Tensor, prec=None, *, m: int | None = None, s: int | None = None,
           workspace: torch.Tensor | None = None, out=None, stream=None, return_info: bool = False):
    """cos(A), sin(A) of a square matrix.

    ``prec``: "fp64", "fp32" or "split_tf32" (default from A's dtype).  A CPU
    tensor is copied to the current device and the results are copied back.
    ``m``/``s`` force the family 2m and the number of double-angle steps.
    """
    p = _prec(prec, A)
    host = not A.is_cuda
    if host:
        A = A.to("cuda", non_blocking=True)
    A = A.contiguous()
    n = _check_matrix(A, p)
    if out is None:
        C = torch.empty_like(A)
        S = torch.empty_like(A)
    else:
        C, S = out
    need = workspace_size(n, p)
    if workspace is None or workspace.numel() * workspace.element_size() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=A.device)
    info = CsInfo()
    fm = -1 if m is None else int(m)
    fs = -1 if s is None else int(s)
    check(lib().cossin_ex(ctypes.c_void_p(A.data_ptr()), n, p, ctypes.c_void_p(C.data_ptr()),
                          ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(workspace.data_ptr()),
                          workspace.numel() * workspace.element_size(), fm, fs, ctypes.byref(info),
                          _stream_ptr(stream)))
    if host:
        C = C.cpu()
        S = S.cpu()
    if return_info:
        return C, S, info.as_dict()
    return C, S


def matmul(X: torch.Tensor, Y: torch.Tensor, prec=None, stream=None) -> torch.Tensor:
    """P = X Y on the library's product kernel for ``prec``."""
    p = _prec(prec, X)
    n = _check_matrix(X, p)
    if _check_matrix(Y, p) != n:
        raise ValueError("X and Y must have the same order")
    P = torch.empty_like(X)
    check(lib().cossin_matmul(ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), n, p,
                              ctypes.c_void_p(P.data_ptr()), _stream_ptr(stream)))
    return P


def prof_enable(on: bool = True) -> None:
    lib().cossin_prof_enable(1 if on else 0)


def prof_reset() -> None:
    lib().cossin_prof_reset()


def prof_read(kind: str):
    """(total ms, launches, algorithmic work) of one kernel kind since the last reset."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    w = ctypes.c_double()
    check(lib().cossin_prof_read(_lib.KERNEL_KINDS[kind], ctypes.byref(ms), ctypes.byref(n), ctypes.byref(w)))
    return ms.value, n.value, w.value
