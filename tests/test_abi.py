"""CPU checks of the C ABI: the library builds, loads and exports every
function declared in include/*.h; host-only calls behave as documented."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import oracle
from paper_2010_00465_gb300 import _lib, api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.add(name)
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert "cossin" in names and "cossin_ex" in names and len(names) >= 9
    for name in names:
        assert hasattr(L, name), name


def test_signatures_cover_header(L):
    for name in declared_functions():
        assert name in _lib.SIGNATURES, name


def test_workspace_size_host_only(L):
    assert api.workspace_size(0, "fp64") > 0
    w64 = api.workspace_size(64, "fp64")
    assert w64 >= 12 * 64 * 64 * 8
    assert api.workspace_size(4096, "fp32") >= 24 * 4096 * 4096 * 4
    with pytest.raises(_lib.CossinError) as e:
        api.workspace_size(-1, "fp64")
    assert e.value.status == _lib.CS_EINVAL
    with pytest.raises(_lib.CossinError):
        api.workspace_size(1 << 20, "fp64")


@pytest.mark.parametrize("table,prec", [(0, "double"), (1, "single")])
def test_select_matches_oracle(L, table, prec):
    for nrm in np.concatenate([[0.0], np.geomspace(1e-8, 1e12, 800)]):
        assert api.select(float(nrm), table) == oracle.select(float(nrm), prec), nrm


def test_select_errors(L):
    for bad, st in ((float("inf"), _lib.CS_ENONFINITE), (float("nan"), _lib.CS_ENONFINITE),
                    (1e300, _lib.CS_ERANGE), (-1.0, _lib.CS_EINVAL)):
        with pytest.raises(_lib.CossinError) as e:
            api.select(bad, 0)
        assert e.value.status == st
    with pytest.raises(_lib.CossinError):
        api.select(1.0, 2)


def test_argument_errors_before_any_gpu_work(L):
    """Checks that fail before the library touches the device."""
    f = L.cossin_ex
    info = _lib.CsInfo()
    nul = ctypes.c_void_p(0)
    assert f(nul, -1, 0, nul, nul, nul, 0, -1, -1, ctypes.byref(info), nul) == _lib.CS_EINVAL
    assert f(nul, 4, 7, nul, nul, nul, 0, -1, -1, ctypes.byref(info), nul) == _lib.CS_EINVAL
    assert f(nul, 4, 0, nul, nul, nul, 0, 24, -1, ctypes.byref(info), nul) == _lib.CS_EINVAL
    assert f(nul, 4, 0, nul, nul, nul, 0, 12, 0, ctypes.byref(info), nul) == _lib.CS_EINVAL
    assert f(nul, 4, 0, nul, nul, nul, 0, 24, 65, ctypes.byref(info), nul) == _lib.CS_EINVAL
    assert f(nul, 4, 0, nul, nul, nul, 0, -1, -1, ctypes.byref(info), nul) == _lib.CS_EINVAL  # null A
    a = ctypes.c_void_p(4096)
    assert f(a, 4, 0, a, ctypes.c_void_p(8192), nul, 0, -1, -1, None, nul) == _lib.CS_EINVAL  # alias
    assert b"overlap" in L.cossin_last_error()
    # n = 0 is a no-op
    assert f(nul, 0, 0, nul, nul, nul, 0, -1, -1, ctypes.byref(info), nul) == _lib.CS_OK


def test_library_has_no_cpu_fallback_symbols(L):
    """The product path has no host implementation of the method to fall back on."""
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    assert "oracle" not in out


def test_emulated_precisions_host_checks(L):
    """The emulated-FP64 precisions add their slice scratch to the workspace
    and accept n <= 8192 only (the int64 level sums), refused before any
    device work."""
    base = {"fp64_emu": "fp64", "split_emu": "split_tf32", "split_bf16": "fp64"}
    for p in ("fp64_emu", "split_emu", "split_bf16"):
        assert api.workspace_size(1024, p) > api.workspace_size(1024, base[p])
        assert api.workspace_size(8192, p) > 0
        with pytest.raises(_lib.CossinError) as e:
            api.workspace_size(8193, p)
        assert e.value.status == _lib.CS_EINVAL
    # the four-slice chain products share the eight-slice scratch
    assert api.workspace_size(1024, "split_bf16") == api.workspace_size(1024, "fp64_emu")
    assert api.workspace_size(8193, "fp64") > 0
    assert api.unitary_workspace_size(100, "fp64") > api.workspace_size(100, "fp64")
    with pytest.raises(_lib.CossinError):
        api.workspace_size(16, 6)
    # the adjoint has no split-precision form
    nul = ctypes.c_void_p(0)
    assert L.cossin_backward_ex(1, 4, nul, nul, nul, nul, nul, nul, -1, -1, _lib.CS_SPLIT_BF16, None,
                                nul) == _lib.CS_EINVAL


def test_adjoint_sizes_that_would_overflow_are_refused(L):
    """count * n^2 beyond 2^46 elements is refused before any device work
    (the byte counts would wrap)."""
    nul = ctypes.c_void_p(0)
    p = ctypes.c_void_p(4096)
    huge = 1 << 40
    assert L.cossin_backward(huge, 4096, p, p, p, p, nul, nul, -1, -1, None, nul) == _lib.CS_EINVAL
    assert b"2^46" in L.cossin_last_error()
    assert L.cossin_unitary_backward(huge, 4096, 1.0, p, p, p, nul, -1, -1, None, nul) == _lib.CS_EINVAL
    assert b"2^46" in L.cossin_last_error()


def test_cs_and_unitary_argument_errors_before_any_gpu_work(L):
    nul = ctypes.c_void_p(0)
    info = _lib.CsInfo()
    cs = L.cossin_cs
    assert cs(nul, 4, float("nan"), 0, nul, nul, nul, 0, -1, -1, ctypes.byref(info), nul) == _lib.CS_EINVAL
    assert cs(nul, 4, 1.0, 0, nul, nul, nul, 0, 4, 0, ctypes.byref(info), nul) == _lib.CS_EINVAL
    assert cs(nul, 4, 1.0, 0, nul, nul, nul, 0, 1, -1, ctypes.byref(info), nul) == _lib.CS_EINVAL
    assert cs(nul, 4, 1.0, 0, nul, nul, nul, 0, 1, 65, ctypes.byref(info), nul) == _lib.CS_EINVAL
    assert cs(nul, 0, 1.0, 0, nul, nul, nul, 0, 2, 3, ctypes.byref(info), nul) == _lib.CS_OK
    assert (info.m, info.s, info.products) == (2, 3, 0)
    un = L.cossin_unitary
    assert un(nul, 4, float("inf"), 0, nul, nul, 0, -1, -1, None, nul) == _lib.CS_EINVAL
    assert un(nul, 0, 1.0, 0, nul, nul, 0, -1, -1, None, nul) == _lib.CS_OK
    ub = L.cossin_unitary_backward
    assert ub(0, 4, 1.0, nul, nul, nul, nul, -1, -1, nul, nul) == _lib.CS_OK
    assert ub(1, 4, float("nan"), nul, nul, nul, nul, -1, -1, nul, nul) == _lib.CS_EINVAL


@pytest.mark.parametrize("table,prec", [(0, "double"), (1, "single")])
def test_cs_select_matches_oracle(L, table, prec):
    """The library's c/s selection (its own theta_cs table) against the oracle's."""
    for nrm in np.concatenate([[0.0], np.geomspace(1e-8, 1e30, 900)]):
        assert api.cs_select(float(nrm), table) == oracle.cs_select(float(nrm), prec), nrm


def test_cs_select_errors(L):
    for bad, st in ((float("inf"), _lib.CS_ENONFINITE), (float("nan"), _lib.CS_ENONFINITE),
                    (1e300, _lib.CS_ERANGE), (-1.0, _lib.CS_EINVAL)):
        with pytest.raises(_lib.CossinError) as e:
            api.cs_select(bad, 0)
        assert e.value.status == st


def test_matmul_argument_errors_before_any_gpu_work(L):
    nul = ctypes.c_void_p(0)
    p = ctypes.c_void_p(4096)
    assert L.cossin_matmul(nul, nul, 0, 0, nul, nul) == _lib.CS_OK  # n = 0: no-op
    assert L.cossin_matmul(nul, nul, -1, 0, nul, nul) == _lib.CS_EINVAL
    assert L.cossin_matmul(p, p, 8, 9, p, nul) == _lib.CS_EINVAL  # unknown precision
    assert L.cossin_matmul(nul, p, 8, 0, ctypes.c_void_p(1 << 20), nul) == _lib.CS_EINVAL  # null X
    assert L.cossin_matmul(p, p, 8, 0, p, nul) == _lib.CS_EINVAL  # P overlaps X
    assert b"overlap" in L.cossin_last_error()
    for prec in (_lib.CS_FP64_EMU, _lib.CS_SPLIT_BF16):
        assert L.cossin_matmul(p, p, 8193, prec, ctypes.c_void_p(1 << 40), nul) == _lib.CS_EINVAL
        assert b"8192" in L.cossin_last_error()


def test_batched_argument_errors_before_any_gpu_work(L):
    size = ctypes.c_size_t()
    ns = (ctypes.c_int64 * 3)(8, 300, 16)
    assert L.cossin_batched_workspace_size(3, ns, ctypes.byref(size)) == _lib.CS_EINVAL
    assert b"256" in L.cossin_last_error()
    ns_ok = (ctypes.c_int64 * 3)(8, 256, 0)
    assert L.cossin_batched_workspace_size(3, ns_ok, ctypes.byref(size)) == _lib.CS_OK and size.value > 0
    big = size.value  # sized by the largest order (per-CTA slices), not by the count
    ns_small = (ctypes.c_int64 * 3)(8, 16, 0)
    assert L.cossin_batched_workspace_size(3, ns_small, ctypes.byref(size)) == _lib.CS_OK and 0 < size.value < big
    assert L.cossin_batched_workspace_size(-1, ns_ok, ctypes.byref(size)) == _lib.CS_EINVAL
    assert L.cossin_batched_workspace_size((1 << 30) + 1, ns_ok, ctypes.byref(size)) == _lib.CS_EINVAL
    assert L.cossin_batched_workspace_size(2, None, ctypes.byref(size)) == _lib.CS_EINVAL
    assert L.cossin_batched_workspace_size(2, ns_ok, None) == _lib.CS_EINVAL


@pytest.mark.parametrize("prec,table", [(_lib.CS_FP64, 0), (_lib.CS_FP64_EMU, 0), (_lib.CS_FP32, 1),
                                        (_lib.CS_SPLIT_TF32, 1), (_lib.CS_SPLIT_EMU, 1), (_lib.CS_SPLIT_BF16, 1)])
def test_precision_selects_its_table(L, prec, table):
    """FP64-accurate kinds use Table 1 (u = 2^-53), the FP32-accurate and
    split kinds Table 2 (u = 2^-24); an n = 0 call reports it without device
    work, for cossin_ex and for cossin_cs."""
    nul = ctypes.c_void_p(0)
    info = _lib.CsInfo()
    assert L.cossin_ex(nul, 0, prec, nul, nul, nul, 0, -1, -1, ctypes.byref(info), nul) == _lib.CS_OK
    assert info.table == table
    info = _lib.CsInfo()
    assert L.cossin_cs(nul, 0, 1.0, prec, nul, nul, nul, 0, -1, -1, ctypes.byref(info), nul) == _lib.CS_OK
    assert info.table == table


def test_backward_workspace_size_host_only(L):
    small = api.backward_workspace_size(4, 64, 0)
    assert small > 4 * 64 * 64 * 8 * 6
    assert api.backward_workspace_size(4, 64, 3) > small          # deeper tape with more double-angle levels
    assert api.backward_workspace_size(8, 64, 3) > api.backward_workspace_size(4, 64, 3)
    assert api.backward_workspace_size(4, 64, 3, "fp64_emu") > api.backward_workspace_size(4, 64, 3)
    assert api.backward_workspace_size(0, 64, 3) == 0
    for bad in (dict(max_s=-1), dict(max_s=65), dict(prec="fp32")):
        kw = dict(count=4, n=64, max_s=3)
        kw.update(bad)
        with pytest.raises(_lib.CossinError) as e:
            api.backward_workspace_size(**kw)
        assert e.value.status == _lib.CS_EINVAL


def test_backward_ws_rejects_missing_workspace(L):
    fake = ctypes.c_void_p(1 << 20)
    st = L.cossin_backward_ws(2, 8, fake, fake, fake, fake, None, None, -1, -1, _lib.CS_FP64, None, 0, None, None)
    assert st == _lib.CS_EINVAL and b"workspace" in L.cossin_last_error()


def test_injected_allocation_failure_returns_enomem(L):
    """The allocation-failure knob: each entry point that allocates returns
    CS_ENOMEM before queuing any work (no GPU is touched here), and the knob
    is used up by exactly the requested number of allocations."""
    a = ctypes.c_void_p(1 << 20)
    c = ctypes.c_void_p(2 << 20)
    s = ctypes.c_void_p(3 << 20)
    api.selftest_fail_next_alloc(4)
    assert L.cossin(a, 64, _lib.CS_FP64, c, s, None) == _lib.CS_ENOMEM
    assert b"cossin workspace" in L.cossin_last_error()
    nrm = ctypes.c_double()
    assert L.cossin_norm1(a, 64, _lib.CS_FP64, ctypes.byref(nrm), None) == _lib.CS_ENOMEM
    assert L.cossin_cs(a, 64, 0.5, _lib.CS_FP64, c, s, None, 0, -1, -1, None, None) == _lib.CS_ENOMEM
    u = ctypes.c_void_p(8 << 20)
    assert L.cossin_unitary(a, 64, 0.5, _lib.CS_FP64, u, None, 0, -1, -1, None, None) == _lib.CS_ENOMEM
    api.selftest_fail_next_alloc(1)
    da = ctypes.c_void_p(16 << 20)
    assert L.cossin_backward(2, 64, a, c, s, da, None, None, -1, -1, None, None) == _lib.CS_ENOMEM
    api.selftest_fail_next_alloc(0)
