"""PyTorch-facing calls of the library.

PyTorch supplies device memory and the current stream; every step of the
method runs in the library's CUDA kernels behind the C ABI.  There is no CPU
fallback: without the built library or a GPU these calls raise.
"""
from __future__ import annotations

import ctypes
import functools
import inspect

import torch

from . import _lib
from ._lib import CsInfo, check, lib

PRECISIONS = {"fp64": _lib.CS_FP64, "fp32": _lib.CS_FP32, "split_tf32": _lib.CS_SPLIT_TF32,
              "fp64_emu": _lib.CS_FP64_EMU, "split_emu": _lib.CS_SPLIT_EMU, "split_bf16": _lib.CS_SPLIT_BF16}
_DTYPE = {_lib.CS_FP64: torch.float64, _lib.CS_FP32: torch.float32, _lib.CS_SPLIT_TF32: torch.float64,
          _lib.CS_FP64_EMU: torch.float64, _lib.CS_SPLIT_EMU: torch.float64, _lib.CS_SPLIT_BF16: torch.float64}


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


def _on_stream(fn):
    """Run the call with its ``stream`` argument (if given) as PyTorch's
    current stream, so that the outputs and workspaces it allocates come from
    that stream's pool: memory freed by work still pending on another stream
    is never handed to a launch on this one."""
    sig = inspect.signature(fn)

    @functools.wraps(fn)
    def wrapper(*args, **kwargs):
        stream = sig.bind_partial(*args, **kwargs).arguments.get("stream")
        if stream is None:
            return fn(*args, **kwargs)
        with torch.cuda.stream(stream):
            return fn(*args, **kwargs)
    return wrapper


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


def device_status(stream=None) -> None:
    """Synchronise ``stream`` and raise CossinError(CS_ETIMEOUT) if a bounded
    wait in a tensor-core kernel expired since the last check (the products
    run asynchronously, so a call's own status covers only its arguments and
    its 1-norm)."""
    check(lib().cossin_device_status(_stream_ptr(stream)))


def workspace_size(n: int, prec="fp64") -> int:
    out = ctypes.c_size_t()
    check(lib().cossin_workspace_size(int(n), _prec(prec), ctypes.byref(out)))
    return int(out.value)


@_on_stream
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


@_on_stream
def cossin(A: torch.Tensor, prec=None, *, m: int | None = None, s: int | None = None,
           workspace: torch.Tensor | None = None, out=None, stream=None, return_info: bool = False,
           check_device: bool = True):
    """cos(A), sin(A) of a square matrix.

    ``prec``: "fp64", "fp32", "split_tf32", "fp64_emu", "split_emu" or
    "split_bf16" (default from A's dtype).  A CPU tensor is copied to the
    current device and the results are copied back: into ``out`` = (C, S) if
    given as CPU tensors (pinned ones are filled by asynchronous copies on the
    call's stream, which is synchronised before returning), else into new CPU
    tensors.  For a device A, ``out`` holds device tensors.  ``m``/``s`` force
    the family 2m and the number of double-angle steps.  With
    ``check_device`` (default) the call synchronises its stream at the end
    and raises if a tensor-core kernel gave up on a bounded wait; without it
    the call returns once the work is queued, and ``device_status`` reports
    such a failure later.
    """
    p = _prec(prec, A)
    host = not A.is_cuda
    host_out = None
    if host:
        if out is not None:
            host_out = out
            for X in host_out:
                if X.is_cuda or X.shape != A.shape or X.dtype != A.dtype or not X.is_contiguous():
                    raise ValueError("host outputs must be contiguous CPU tensors shaped and typed like A")
            out = None
        # on the call's stream; asynchronous only from pinned memory (a copy
        # from pageable memory blocks until the data is on the device)
        A = A.to("cuda", non_blocking=A.is_pinned())
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
    if check_device:
        device_status(stream)
    if host:
        if host_out is not None:
            host_out[0].copy_(C, non_blocking=host_out[0].is_pinned())
            host_out[1].copy_(S, non_blocking=host_out[1].is_pinned())
            torch.cuda.current_stream().synchronize()
            C, S = host_out
        else:
            C = C.cpu()
            S = S.cpu()
    if return_info:
        return C, S, info.as_dict()
    return C, S


def cs_select(normB: float, table: int):
    """(family, sigma) that cossin_cs takes for ||t^2 A||_1 = normB; table 0 = double, 1 = single."""
    f = ctypes.c_int32()
    sg = ctypes.c_int32()
    check(lib().cossin_cs_select(float(normB), int(table), ctypes.byref(f), ctypes.byref(sg)))
    return f.value, sg.value


@_on_stream
def cossin_cs(A: torch.Tensor, t: float, prec=None, *, family: int | None = None, sigma: int | None = None,
              workspace: torch.Tensor | None = None, out=None, stream=None, return_info: bool = False,
              check_device: bool = True):
    """c(t^2 A) = cos(sqrt(t^2 A)) and s(t, A) = A^(-1/2) sin(sqrt(t^2 A)) (Sec. 2.2).

    ``family`` (0..3: 2, 3, 4 or 5 products) and ``sigma`` (double-angle
    steps) force the scheme; info["m"] is the family, info["norm1"] ||t^2 A||_1.
    ``check_device`` as for ``cossin``.
    """
    p = _prec(prec, A)
    host = not A.is_cuda
    if host:
        A = A.to("cuda", non_blocking=A.is_pinned())
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
    ff = -1 if family is None else int(family)
    fs = -1 if sigma is None else int(sigma)
    check(lib().cossin_cs(ctypes.c_void_p(A.data_ptr()), n, float(t), p, ctypes.c_void_p(C.data_ptr()),
                          ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(workspace.data_ptr()),
                          workspace.numel() * workspace.element_size(), ff, fs, ctypes.byref(info),
                          _stream_ptr(stream)))
    if check_device:
        device_status(stream)
    if host:
        C = C.cpu()
        S = S.cpu()
    if return_info:
        return C, S, info.as_dict()
    return C, S


@_on_stream
def matmul(X: torch.Tensor, Y: torch.Tensor, prec=None, stream=None) -> torch.Tensor:
    """P = X Y on the library's product kernel for ``prec``."""
    p = _prec(prec, X)
    n = _check_matrix(X, p)
    if _check_matrix(Y, p) != n:
        raise ValueError("X and Y must have the same order")
    P = torch.empty_like(X)
    check(lib().cossin_matmul(ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), n, p,
                              ctypes.c_void_p(P.data_ptr()), _stream_ptr(stream)))
    device_status(stream)
    return P


@_on_stream
def cossin_backward(A: torch.Tensor, G_C: torch.Tensor, G_S: torch.Tensor, *, m: int | None = None,
                    s: int | None = None, want_forward: bool = False, stream=None, return_info: bool = False,
                    prec: str = "fp64", workspace: torch.Tensor | None = None):
    """Gradient of <G_C, cos(A)> + <G_S, sin(A)> (FP64; A is n x n or a
    [count, n, n] batch), at the (2m, s) the forward pass uses.  ``prec``
    "fp64_emu" emulates the FP64 products on the BF16 tensor cores.  With a
    ``workspace`` (uint8 CUDA tensor of at least backward_workspace_size
    bytes for the largest s the inputs select) the library allocates
    nothing."""
    import numpy as np
    if A.dtype != torch.float64 or G_C.dtype != torch.float64 or G_S.dtype != torch.float64:
        raise TypeError("the adjoint runs in FP64")
    batched = A.dim() == 3
    A3 = A if batched else A.unsqueeze(0)
    if A3.shape[-1] != A3.shape[-2]:
        raise ValueError("square matrices expected")
    A3 = A3.contiguous()
    GC3 = (G_C if batched else G_C.unsqueeze(0)).contiguous()
    GS3 = (G_S if batched else G_S.unsqueeze(0)).contiguous()
    if GC3.shape != A3.shape or GS3.shape != A3.shape:
        raise ValueError("cotangents must match A")
    for T in (A3, GC3, GS3):
        if not T.is_cuda:
            raise ValueError("CUDA tensors expected")
    count, n = A3.shape[0], A3.shape[1]
    dA = torch.empty_like(A3)
    C = torch.empty_like(A3) if want_forward else None
    S = torch.empty_like(A3) if want_forward else None
    infos = (CsInfo * max(count, 1))()
    fm = -1 if m is None else int(m)
    fs = -1 if s is None else int(s)
    ptrs = (count, n, ctypes.c_void_p(A3.data_ptr()), ctypes.c_void_p(GC3.data_ptr()),
            ctypes.c_void_p(GS3.data_ptr()), ctypes.c_void_p(dA.data_ptr()),
            ctypes.c_void_p(C.data_ptr() if C is not None else 0),
            ctypes.c_void_p(S.data_ptr() if S is not None else 0), fm, fs, _prec(prec))
    if workspace is None:
        check(lib().cossin_backward_ex(*ptrs, infos, _stream_ptr(stream)))
    else:
        if not workspace.is_cuda:
            raise ValueError("the workspace must be a CUDA tensor")
        check(lib().cossin_backward_ws(*ptrs, ctypes.c_void_p(workspace.data_ptr()),
                                       workspace.numel() * workspace.element_size(), infos, _stream_ptr(stream)))
    device_status(stream)
    if not batched:
        dA = dA[0]
        C = C[0] if C is not None else None
        S = S[0] if S is not None else None
    out = (dA, C, S) if want_forward else dA
    if return_info:
        return out, [infos[i].as_dict() for i in range(count)]
    return out


def backward_workspace_size(count: int, n: int, max_s: int, prec: str = "fp64") -> int:
    """Bytes of the caller workspace of cossin_backward for ``count`` matrices
    of order n whose (2m, s) have s <= max_s."""
    out = ctypes.c_size_t()
    check(lib().cossin_backward_workspace_size(int(count), int(n), _prec(prec), int(max_s), ctypes.byref(out)))
    return int(out.value)


def fp64_fma_rate(rounds: int = 16384, stream=None) -> float:
    """Measured FP64 FMA throughput of the current device, TFLOP/s."""
    out = ctypes.c_double()
    check(lib().cossin_fp64_fma_rate(int(rounds), ctypes.byref(out), _stream_ptr(stream)))
    return float(out.value)


def fp64_product_launches(M: int, N: int, K: int) -> int:
    """Kernels one FP64 product (M x N result, inner K) launches inside cossin
    on the current device: 2 when its last partial wave of tiles is split
    over K, else 1."""
    out = ctypes.c_int32()
    check(lib().cossin_fp64_product_launches(int(M), int(N), int(K), ctypes.byref(out)))
    return int(out.value)


def selftest_fail_next_alloc(count: int = 1) -> None:
    """Test hook: the library's next ``count`` device allocations fail (CS_ENOMEM)."""
    lib().cossin_selftest_fail_next_alloc(int(count))


def unitary_workspace_size(n: int, prec="fp64") -> int:
    out = ctypes.c_size_t()
    check(lib().cossin_unitary_workspace_size(int(n), _prec(prec), ctypes.byref(out)))
    return out.value


@_on_stream
def unitary(A: torch.Tensor, t: float, prec=None, *, m: int | None = None, s: int | None = None,
            workspace: torch.Tensor | None = None, stream=None, return_info: bool = False):
    """U = exp(-i t A) = cos(tA) - i sin(tA) of a real square matrix (complex64
    for "fp32", complex128 for every other precision)."""
    p = _prec(prec, A)
    A = A.contiguous()
    n = _check_matrix(A, p)
    U = torch.empty((n, n), dtype=torch.complex64 if p == _lib.CS_FP32 else torch.complex128, device=A.device)
    need = unitary_workspace_size(n, p)
    if workspace is None or workspace.numel() * workspace.element_size() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=A.device)
    info = CsInfo()
    fm = -1 if m is None else int(m)
    fs = -1 if s is None else int(s)
    check(lib().cossin_unitary(ctypes.c_void_p(A.data_ptr()), n, float(t), p, ctypes.c_void_p(U.data_ptr()),
                               ctypes.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size(),
                               fm, fs, ctypes.byref(info), _stream_ptr(stream)))
    device_status(stream)
    return (U, info.as_dict()) if return_info else U


@_on_stream
def unitary_backward(A: torch.Tensor, t: float, G: torch.Tensor, *, m: int | None = None, s: int | None = None,
                     want_forward: bool = False, stream=None, return_info: bool = False):
    """d/dA of Re sum(conj(G) * exp(-i t A)) (FP64; A real n x n or [count, n, n],
    G complex128 of the same shape)."""
    if A.dtype != torch.float64 or G.dtype != torch.complex128:
        raise TypeError("the unitary adjoint takes a float64 A and a complex128 G")
    batched = A.dim() == 3
    A3 = (A if batched else A.unsqueeze(0)).contiguous()
    G3 = (G if batched else G.unsqueeze(0)).contiguous()
    if A3.shape[-1] != A3.shape[-2] or G3.shape != A3.shape:
        raise ValueError("square A and a G of the same shape expected")
    if not (A3.is_cuda and G3.is_cuda):
        raise ValueError("CUDA tensors expected")
    count, n = A3.shape[0], A3.shape[1]
    dA = torch.empty_like(A3)
    U = torch.empty_like(G3) if want_forward else None
    infos = (CsInfo * max(count, 1))()
    fm = -1 if m is None else int(m)
    fs = -1 if s is None else int(s)
    check(lib().cossin_unitary_backward(count, n, float(t), ctypes.c_void_p(A3.data_ptr()),
                                        ctypes.c_void_p(G3.data_ptr()), ctypes.c_void_p(dA.data_ptr()),
                                        ctypes.c_void_p(U.data_ptr() if U is not None else 0), fm, fs, infos,
                                        _stream_ptr(stream)))
    if not batched:
        dA = dA[0]
        U = U[0] if U is not None else None
    out = (dA, U) if want_forward else dA
    if return_info:
        return out, [infos[i].as_dict() for i in range(count)]
    return out


class Unitary(torch.autograd.Function):
    """exp(-i t A) for a real FP64 n x n A, with the library's adjoint as backward
    (gradient with respect to A; t is a constant)."""

    @staticmethod
    def forward(ctx, A, t):
        ctx.save_for_backward(A)
        ctx.t = float(t)
        return unitary(A, t, "fp64")

    @staticmethod
    def backward(ctx, gU):
        (A,) = ctx.saved_tensors
        return unitary_backward(A, ctx.t, gU.contiguous()), None


def unitary_autograd(A: torch.Tensor, t: float):
    return Unitary.apply(A, t)


class CosSin(torch.autograd.Function):
    """(cos A, sin A) with the library's adjoint as backward (FP64; A is n x n
    or a [count, n, n] batch).  The backward recomputes the forward pass with
    its product operands kept, at the same (2m, s)."""

    @staticmethod
    def forward(ctx, A):
        if A.dim() == 2:
            C, S = cossin(A, "fp64")
        else:
            outs = [cossin(a, "fp64") for a in A]
            C = torch.stack([o[0] for o in outs])
            S = torch.stack([o[1] for o in outs])
        ctx.save_for_backward(A)
        return C, S

    @staticmethod
    def backward(ctx, gC, gS):
        (A,) = ctx.saved_tensors
        gC = torch.zeros_like(A) if gC is None else gC.contiguous()
        gS = torch.zeros_like(A) if gS is None else gS.contiguous()
        return cossin_backward(A, gC, gS)


def cossin_autograd(A: torch.Tensor):
    return CosSin.apply(A)


INFO_DTYPE = None


def _info_dtype():
    import numpy as np
    return np.dtype([("norm1", "<f8"), ("m", "<i4"), ("s", "<i4"), ("products", "<i4"), ("table", "<i4"),
                     ("flops", "<f8")])


class BatchedPlan:
    """cos/sin of a list of square FP32 CUDA matrices (orders <= 256), each with
    its own (2m, s), as one persistent launch replayed from a CUDA graph.

    ``launch()`` recomputes every matrix from the current contents of the
    inputs; results land in ``self.C`` / ``self.S``; ``infos()`` and
    ``status()`` read the per-matrix record of the last launch."""

    @_on_stream
    def __init__(self, mats, autotune: bool = True, stream=None, out=None):
        import numpy as np
        self.A = list(mats)
        for A in self.A:
            _check_matrix(A, _lib.CS_FP32)
        count = len(self.A)
        self.count = count
        self.n = np.array([A.shape[0] for A in self.A], dtype=np.int64)
        if out is None:
            self.C = [torch.empty_like(A) for A in self.A]
            self.S = [torch.empty_like(A) for A in self.A]
        else:
            self.C, self.S = out
        dev = self.A[0].device if count else torch.device("cuda")
        self._pa = (ctypes.c_void_p * max(count, 1))(*[A.data_ptr() for A in self.A])
        self._pc = (ctypes.c_void_p * max(count, 1))(*[C.data_ptr() for C in self.C])
        self._ps = (ctypes.c_void_p * max(count, 1))(*[S.data_ptr() for S in self.S])
        size = ctypes.c_size_t()
        check(lib().cossin_batched_workspace_size(count, self.n.ctypes.data, ctypes.byref(size)))
        self.ws = torch.empty(max(size.value, 1), dtype=torch.uint8, device=dev)
        self._infos = torch.zeros(max(count, 1) * 32, dtype=torch.uint8, device=dev)
        self._status = torch.zeros(max(count, 1), dtype=torch.int32, device=dev)
        self._plan = ctypes.c_void_p()
        check(lib().cossin_batched_plan_create(
            count, self.n.ctypes.data, self._pa, self._pc, self._ps, ctypes.c_void_p(self.ws.data_ptr()),
            self.ws.numel(), ctypes.c_void_p(self._infos.data_ptr()), ctypes.c_void_p(self._status.data_ptr()),
            1 if autotune else 0, _stream_ptr(stream), ctypes.byref(self._plan)))

    def launch(self, stream=None):
        check(lib().cossin_batched_plan_launch(self._plan, _stream_ptr(stream)))
        return self.C, self.S

    def variant(self):
        t = ctypes.c_int32()
        c = ctypes.c_int32()
        check(lib().cossin_batched_plan_info(self._plan, ctypes.byref(t), ctypes.byref(c)))
        return {"tile": t.value, "ctas_per_sm": c.value}

    def infos(self):
        import numpy as np
        raw = self._infos.cpu().numpy().tobytes()[: 32 * self.count]
        return np.frombuffer(raw, dtype=_info_dtype())

    def status(self):
        return self._status[: self.count].cpu().numpy()

    def close(self):
        if getattr(self, "_plan", None) and self._plan.value:
            lib().cossin_batched_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@_on_stream
def cossin_batched(mats, stream=None):
    """One-shot batched cos/sin (no graph); returns (C list, S list, infos, status)."""
    import numpy as np
    mats = list(mats)
    for A in mats:
        _check_matrix(A, _lib.CS_FP32)
    count = len(mats)
    n = np.array([A.shape[0] for A in mats], dtype=np.int64)
    C = [torch.empty_like(A) for A in mats]
    S = [torch.empty_like(A) for A in mats]
    pa = (ctypes.c_void_p * max(count, 1))(*[A.data_ptr() for A in mats])
    pc = (ctypes.c_void_p * max(count, 1))(*[X.data_ptr() for X in C])
    ps = (ctypes.c_void_p * max(count, 1))(*[X.data_ptr() for X in S])
    size = ctypes.c_size_t()
    check(lib().cossin_batched_workspace_size(count, n.ctypes.data, ctypes.byref(size)))
    dev = mats[0].device if count else torch.device("cuda")
    ws = torch.empty(max(size.value, 1), dtype=torch.uint8, device=dev)
    infos = torch.zeros(max(count, 1) * 32, dtype=torch.uint8, device=dev)
    status = torch.zeros(max(count, 1), dtype=torch.int32, device=dev)
    check(lib().cossin_batched(count, n.ctypes.data, pa, pc, ps, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                               ctypes.c_void_p(infos.data_ptr()), ctypes.c_void_p(status.data_ptr()),
                               _stream_ptr(stream)))
    inf = np.frombuffer(infos.cpu().numpy().tobytes()[: 32 * count], dtype=_info_dtype())
    return C, S, inf, status[:count].cpu().numpy()


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
