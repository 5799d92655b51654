"""Parity of the batched FP32 path (one persistent launch, per-matrix (2m, s))
with the FP64 oracle run per matrix on the same FP32 input with the single
table at the same (2m, s)."""
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
    den = np.linalg.norm(Y)
    return float(np.linalg.norm(X - Y) / den) if den > 0 else float(np.linalg.norm(X - Y))


def check_against_oracle(A32, C, S, info):
    A = A32.astype(np.float64)
    nrm = oracle.norm1(A)
    assert info["norm1"] == pytest.approx(nrm, rel=1e-13, abs=0.0)
    assert (int(info["m"]), int(info["s"])) == oracle.select(nrm, "single")
    Co, So, _ = oracle.cossin(A, "single", m=int(info["m"]), s=int(info["s"]))
    t = TOL32
    ec, es = relfro(C, Co), relfro(S, So)
    assert ec <= t and es <= t, (A.shape[0], nrm, ec, es)


def make_batch(count, index, **kw):
    mats, ns, norms = inputs.batch(count, index=index, **kw)
    dev = [torch.from_numpy(M).cuda() for M in mats]
    return mats, dev


@pytest.mark.parametrize("autotune", [False, True])
def test_small_mixed_batch(autotune):
    mats, dev = make_batch(48, index=80)
    plan = api.BatchedPlan(dev, autotune=autotune)
    plan.launch()
    torch.cuda.synchronize()
    infos = plan.infos()
    assert np.all(plan.status() == 0)
    for k in range(len(mats)):
        check_against_oracle(mats[k], plan.C[k].cpu().numpy(), plan.S[k].cpu().numpy(), infos[k])
    assert plan.variant()["tile"] in (64, 128)


def test_one_shot_entry_point():
    mats, dev = make_batch(20, index=81, n_lo=1, n_hi=200)
    C, S, infos, status = api.cossin_batched(dev)
    torch.cuda.synchronize()
    assert np.all(status == 0)
    for k in range(len(mats)):
        check_against_oracle(mats[k], C[k].cpu().numpy(), S[k].cpu().numpy(), infos[k])


def test_every_order_and_family():
    """Orders 1..256 including every tile edge, both tile shapes."""
    ns = [1, 2, 3, 7, 8, 15, 16, 17, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129, 200, 255, 256]
    fams = ["normal", "symmetric", "triangular", "uniform01", "nilpotent", "uniform_pm"]
    mats = []
    for i, n in enumerate(ns):
        nrm = [2.0 ** -6, 0.3, 1.0, 4.0, 8.0, 30.0, 64.0][i % 7]
        mats.append(inputs.matrix(n, fams[i % len(fams)], nrm if n > 1 else 0.5, index=82, sub=i).astype(np.float32))
    dev = [torch.from_numpy(M).cuda() for M in mats]
    plan = api.BatchedPlan(dev, autotune=True)
    plan.launch()
    torch.cuda.synchronize()
    infos = plan.infos()
    for k in range(len(mats)):
        check_against_oracle(mats[k], plan.C[k].cpu().numpy(), plan.S[k].cpu().numpy(), infos[k])


def test_order_norm_grid():
    """Orders {1, 5, 33, 64, 129, 192, 256} x ||A||_1 {8, 30, 64}, normal and
    symmetric: every FP32-class result within 2e-5 of the oracle."""
    mats = []
    for fam in ("normal", "symmetric"):
        for n in (1, 5, 33, 64, 129, 192, 256):
            for nrm in (8.0, 30.0, 64.0):
                mats.append(inputs.matrix(n, fam, nrm, index=86, sub=n).astype(np.float32))
    dev = [torch.from_numpy(M).cuda() for M in mats]
    plan = api.BatchedPlan(dev, autotune=False)
    plan.launch()
    torch.cuda.synchronize()
    infos = plan.infos()
    assert np.all(plan.status() == 0)
    for k in range(len(mats)):
        check_against_oracle(mats[k], plan.C[k].cpu().numpy(), plan.S[k].cpu().numpy(), infos[k])


def test_replay_recomputes_and_is_deterministic():
    mats, dev = make_batch(30, index=83)
    plan = api.BatchedPlan(dev, autotune=False)
    plan.launch()
    torch.cuda.synchronize()
    C1 = [c.clone() for c in plan.C]
    plan.launch()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(C1, plan.C))
    for A in dev:
        A.mul_(0.5)
    plan.launch()
    torch.cuda.synchronize()
    infos = plan.infos()
    for k in range(len(mats)):
        check_against_oracle(mats[k] * np.float32(0.5), plan.C[k].cpu().numpy(), plan.S[k].cpu().numpy(), infos[k])


def test_error_status_per_matrix():
    good = inputs.matrix(20, "normal", 2.0, index=84).astype(np.float32)
    bad = good.copy()
    bad[3, 4] = np.nan
    huge = np.full((5, 5), 1e30, dtype=np.float32)
    zero = np.zeros((0, 0), dtype=np.float32)
    dev = [torch.from_numpy(M).cuda() for M in (good, bad, huge, zero, good)]
    C, S, infos, status = api.cossin_batched(dev)
    torch.cuda.synchronize()
    assert list(status) == [_lib.CS_OK, _lib.CS_ENONFINITE, _lib.CS_ERANGE, _lib.CS_OK, _lib.CS_OK]
    assert torch.isnan(C[1]).all() and torch.isnan(S[2]).all()
    check_against_oracle(good, C[0].cpu().numpy(), S[0].cpu().numpy(), infos[0])
    assert torch.equal(C[0], C[4])


def test_rejects_large_orders():
    A = torch.zeros(257, 257, device="cuda")
    with pytest.raises(_lib.CossinError) as ex:
        api.cossin_batched([A])
    assert ex.value.status == _lib.CS_EINVAL


def test_full_workload_sampled():
    """20,000 FP32 matrices, n log-uniform in [8, 256], ||A||_1 log-uniform in
    [2^-6, 2^6], half symmetric: one graph-captured persistent launch; a
    sample of matrices (the largest, the smallest and a random set) is checked
    against the oracle one by one, the rest through their recorded norms."""
    count = 20000
    ns, norms, fams = inputs.batch_shapes(count, index=3)
    g = inputs.rng(3, 99)
    flat = []
    sample = (set(np.argsort(-ns)[:4]) | set(np.argsort(ns)[:4]) | set(np.argsort(-norms)[:8])
              | set(g.choice(count, 24, replace=False)))
    mats_np = {}
    for i in range(count):
        M = inputs.matrix(int(ns[i]), str(fams[i]), float(norms[i]), index=3, sub=i + 1).astype(np.float32)
        if i in sample:
            mats_np[i] = M
        flat.append(torch.from_numpy(M))
    dev = [t.cuda() for t in flat]
    plan = api.BatchedPlan(dev, autotune=True)
    plan.launch()
    torch.cuda.synchronize()
    assert np.all(plan.status() == 0)
    infos = plan.infos()
    got_norms = infos["norm1"]
    want_norms = np.array([float(np.abs(t.numpy().astype(np.float64)).sum(axis=0).max()) for t in flat])
    assert np.allclose(got_norms, want_norms, rtol=1e-12, atol=0)
    for i in sorted(sample):
        check_against_oracle(mats_np[i], plan.C[i].cpu().numpy(), plan.S[i].cpu().numpy(), infos[i])
