"""Mixed-precision refinement (FP32 / BF16 block storage, FP32 sweeps, FP64
residual and update) against the FP64 oracle.

Tolerances:
  * one outer step (K correction sweeps from d = 0, then pi <- (pi+d)/e^T(pi+d))
    against the oracle's step with the operators quantized exactly as stored
    (FP32, or BF16 with a power-of-two scale per block) and FP64 arithmetic:
    relative L1 <= 2e-6 for both storage types (what remains is the FP32
    arithmetic and the FP32 correction vector: about 2^-24 per operation, sums
    of same-sign terms, K = 12 sweeps); against the unquantized FP64 step the
    storage rounding itself shows: <= 2e-6 (FP32) and <= 2e-2 (BF16, 2^-9 per
    entry);
  * full solves to ||Q^T pi||_1 <= 1e-12: relative L1 <= 1e-10 against the
    FP64 oracle's solution (the FP64 residual decides convergence).
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

mc = pytest.importorskip("paper_2302_07551_gb300")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_l1(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).sum() / np.abs(np.asarray(b)).sum()


@pytest.mark.parametrize("dtype,tol", [("f32", 2e-6), ("bf16", 2e-2)])
@pytest.mark.parametrize("apply", ["inverse", "coupled"])
@pytest.mark.parametrize("L,m,stair", [(40, 64, 1), (13, 256, 1), (9, 128, 2), (30, 12, 1),
                                        (7, 132, 1), (11, 200, 2), (21, 40, 2), (17, 36, 1),
                                        (5, 8, 1), (19, 16, 1), (10, 32, 2), (12, 20, 1)])
def test_one_refinement_step(L, m, stair, apply, dtype, tol):
    K = 12
    blocks = synth.qbd(L, m, 0.85, seed=L + m)
    oc = oracle.Chain(*blocks)
    meth = oracle.STAIR1 if stair == 1 else oracle.STAIR2
    N = L * m
    pi0 = np.full(N, 1.0 / N)
    r = oc.residual_vec(pi0)
    d = np.zeros(N)
    for _ in range(K):
        d = oc.sweep_rhs(d, -r, meth)
    ref = (pi0 + d) / (pi0 + d).sum()
    qref = oc.refinement_step(pi0, K, dtype, apply, meth)
    ch = mc.Chain(*(dev(b) for b in blocks), stair=stair, apply=apply, dtype=dtype)
    pi, res = ch.solve(tol=0.0, maxit=K, check_every=K)
    got = pi.cpu().numpy()
    assert res["sweeps"] == K
    assert rel_l1(got, qref) <= 2e-6, rel_l1(got, qref)
    assert rel_l1(got, ref) <= tol, rel_l1(got, ref)
    # the reported residual is the FP64 residual of the returned iterate
    assert abs(res["residual"] - oc.residual(got)) <= 1e-9 * oc.residual(got)
    ch.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("apply", ["inverse", "coupled"])
def test_refined_solution_matches_fp64_oracle(dtype, apply):
    L, m = 48, 64
    blocks = synth.qbd(L, m, 0.85, seed=3)
    oc = oracle.Chain(*blocks)
    ref = oc.solve(tol=1e-13, maxit=200000, check_every=50)
    ch = mc.Chain(*(dev(b) for b in blocks), apply=apply, dtype=dtype)
    pi, res = ch.solve(tol=1e-12, maxit=200000, check_every=64)
    got = pi.cpu().numpy()
    assert res["converged"] and res["residual"] <= 1e-12
    assert rel_l1(got, ref["x"]) <= 1e-10
    assert abs(got.sum() - 1.0) <= 1e-13 and got.min() >= -1e-30
    # the residual reported is the oracle's residual of the same vector
    assert abs(oc.residual(got) - res["residual"]) <= 1e-3 * res["residual"] + 1e-16
    ch.close()


def test_low_precision_needs_m_multiple_of_4():
    blocks = synth.qbd(8, 6, 0.85, seed=1)
    with pytest.raises(ValueError):
        mc.Chain(*(dev(b) for b in blocks), dtype="bf16")


@pytest.mark.parametrize("dtype,apply,m", [("bf16", "coupled", 64), ("f32", "inverse", 64),
                                           ("bf16", "inverse", 128), ("bf16", "coupled", 16),
                                           ("f64", "inverse", 64)])
def test_tuning_changes_no_result(dtype, apply, m):
    """mc_tune picks a launch configuration (blocks per SM, levels per claimed
    unit) by timing; every configuration gives bitwise the same iterates, and
    a solve after tuning still matches the oracle."""
    L = 150
    blocks = synth.qbd(L, m, 0.8, seed=60 + m, level_dependent=True)
    ch = mc.Chain(*(torch.from_numpy(b).cuda() for b in blocks), dtype=dtype, apply=apply)
    N = L * m
    x = torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda")
    ref, _ = ch.solve(tol=0.0, maxit=96, check_every=32)
    bps, lpu, ms = ch.tune(x, 32)
    assert ms > 0 and bps >= 0 and lpu in (1, 2, 4)
    assert ch.tuning() == (bps, lpu)
    cands = [(0, 1), (2, 2), (3, 4)] if dtype != "f64" else [(0, 1), (1, 1), (2, 1)]
    for b, u in cands:
        ch.set_tuning(b, u)
        out, _ = ch.solve(tol=0.0, maxit=96, check_every=32)
        assert torch.equal(out, ref), (b, u)
    if dtype == "f64":
        with pytest.raises(mc.McError):
            ch.set_tuning(0, 2)          # FP64 sweeps take one level per unit
    ch.set_tuning(bps, lpu)
    pi, res = ch.solve(tol=1e-12, maxit=400000, check_every=32)
    sol = oracle.Chain(*blocks).solve(tol=1e-13, maxit=400000, check_every=32)["x"]
    assert res["converged"] and np.abs(pi.cpu().numpy() - sol).sum() / np.abs(sol).sum() <= 1e-10
    ch.close()
