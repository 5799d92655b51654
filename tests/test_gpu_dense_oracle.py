"""Dense full-size parity with the oracle, element by element.

One dense N(0,1) matrix of order 2304 at ||A||_1 = 64 (FP32-representable
entries, so every precision gets the same input).  At this order the native
FP64 product switches to its 128-wide tiles and every tensor-core kernel runs
many tiles with a ragged K tail (2304 = 18 x 128), and the long-K accumulation
of every product is checked against the oracle's plain triple loops, which
the block-diagonal n = 4096 cases (64 non-zeros per dot product) do not do.
The FP64-class precisions are compared with the oracle's double-table result
at 1e-11, the FP32 class with its single-table result at 2e-5 (relative
Frobenius), each at the oracle's (2m, s).  The two oracle evaluations take
about a minute on the host cores and are shared by the module.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2010_00465_gb300 import api, inputs

pytestmark = pytest.mark.gpu
N = 2304


def relfro(X, Y):
    X = np.asarray(X, dtype=np.float64)
    return float(np.linalg.norm(X - Y) / np.linalg.norm(Y))


@pytest.fixture(scope="module")
def case():
    A = inputs.matrix(N, "normal", 64.0, index=70).astype(np.float32).astype(np.float64)
    Cd, Sd, id_ = oracle.cossin(A, "double")
    Cs, Ss, is_ = oracle.cossin(A, "single")
    return A, (Cd, Sd, id_), (Cs, Ss, is_)


@pytest.mark.parametrize("prec", ["fp64", "fp64_emu"])
def test_fp64_class_dense_2304(case, prec):
    A, (Co, So, io), _ = case
    assert (io["m"], io["s"]) == (24, 6)
    C, S, info = api.cossin(torch.from_numpy(A).cuda(), prec, return_info=True)
    assert (info["m"], info["s"]) == (io["m"], io["s"])
    assert info["norm1"] == pytest.approx(io["norm1"], rel=1e-14)
    ec, es = relfro(C.cpu().numpy(), Co), relfro(S.cpu().numpy(), So)
    assert ec <= 1e-11 and es <= 1e-11, (prec, ec, es)


@pytest.mark.parametrize("prec", ["fp32", "split_tf32", "split_emu", "split_bf16"])
def test_fp32_class_dense_2304(case, prec):
    A, _, (Co, So, io) = case
    assert (io["m"], io["s"]) == (24, 4)
    dt = torch.float32 if prec == "fp32" else torch.float64
    C, S, info = api.cossin(torch.from_numpy(A).to("cuda", dt), prec, return_info=True)
    assert (info["m"], info["s"], info["table"]) == (io["m"], io["s"], 1)
    ec, es = relfro(C.double().cpu().numpy(), Co), relfro(S.double().cpu().numpy(), So)
    assert ec <= 2e-5 and es <= 2e-5, (prec, ec, es)
